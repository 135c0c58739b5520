// Sec. 3.4 outlier filtering and Sec. 3.5 sparsification.
//
//   consistency  Eq. 5 two-way check against two backward flows; per pixel.
//   region       connected components of the surviving pixels (4-neighbours with
//                flow difference below 3 px) by lock-free union-find: a link
//                always hangs the larger root under the smaller one with one
//                atomicCAS, so every component's root is its smallest pixel index
//                and the labelling is unique. Components smaller than s that touch
//                a consistency-rejected neighbour within 3 px are removed.
//   sparsify     one pixel per aligned 3x3 block with >= e survivors (smallest
//                sum of the two consistency errors, raster-first on ties),
//                compacted in block raster order (per-CTA counts, their scan, then
//                ranked writes: deterministic).
// Flows are in units of 1/q pixel (q = 2^lq; q = 1: pixels): thresholds scale
// by q, and a subpixel target reads the backward flows at its nearest pixel.
#include "ff_internal.cuh"

namespace ff {

__device__ __forceinline__ bool close3(uint32_t a, uint32_t b, int lq) {
  const int dx = flow_dx(a) - flow_dx(b), dy = flow_dy(a) - flow_dy(b);
  return dx * dx + dy * dy < (9 << (2 * lq));
}

// The pixel nearest to the target of flow f at pixel (x, y) (halves rounded up).
__device__ __forceinline__ void target_pixel(int x, int y, uint32_t f, int lq, int &qx, int &qy) {
  const int half = (1 << lq) >> 1;
  qx = ((x << lq) + flow_dx(f) + half) >> lq;  // arithmetic shift: floor
  qy = ((y << lq) + flow_dy(f) + half) >> lq;
}

__global__ void k_consistency(const uint32_t *__restrict__ F, const uint32_t *__restrict__ Fb1,
                              const uint32_t *__restrict__ Fb2, int W, int H, int eps, int lq,
                              uint8_t *__restrict__ vcc, int32_t *__restrict__ err,
                              int32_t *__restrict__ parent) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= W * H) return;
  const int x = p % W, y = p / W;
  const uint32_t f = F[p];
  int qx, qy;
  target_pixel(x, y, f, lq, qx, qy);
  uint8_t ok = 0;
  int32_t es = 0x7fffffff;
  if (qx >= 0 && qx < W && qy >= 0 && qy < H) {
    const int q = qy * W + qx;
    const uint32_t b1 = Fb1[q], b2 = Fb2[q];
    const long long a0 = flow_dx(f) + flow_dx(b1), a1 = flow_dy(f) + flow_dy(b1);
    const long long c0 = flow_dx(f) + flow_dx(b2), c1 = flow_dy(f) + flow_dy(b2);
    const long long epsq = (long long)eps << lq;
    const long long e1 = a0 * a0 + a1 * a1, e2 = c0 * c0 + c1 * c1, e2eps = epsq * epsq;
    ok = (e1 < e2eps) && (e2 < e2eps);
    es = (int32_t)min(e1 + e2, (long long)0x7fffffff);
  }
  vcc[p] = ok;
  err[p] = es;
  parent[p] = ok ? p : -1;
}

// Root of x with path halving. Every parent index is smaller than its child's
// and only roots are ever relinked (by atomicCAS in uf_unite), so pointing a
// non-root at its grandparent keeps it inside its set and is safe to race.
__device__ __forceinline__ int uf_find(int32_t *parent, int x) {
  int p = parent[x];
  while (p != x) {
    const int g = parent[p];
    if (g != p) parent[x] = g;
    x = p;
    p = g;
  }
  return x;
}

__device__ void uf_unite(int32_t *parent, int a, int b) {
  while (true) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicCAS(&parent[b], b, a);
    if (old == b) return;
    b = old;
  }
}

__global__ void k_union(const uint32_t *__restrict__ F, const uint8_t *__restrict__ vcc, int W, int H,
                        int lq, int32_t *parent) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= W * H || !vcc[p]) return;
  const int x = p % W, y = p / W;
  const uint32_t f = F[p];
  if (x + 1 < W && vcc[p + 1] && close3(f, F[p + 1], lq)) uf_unite(parent, p, p + 1);
  if (y + 1 < H && vcc[p + W] && close3(f, F[p + W], lq)) uf_unite(parent, p, p + W);
}

// Root without compression. In k_flatten each thread stores the root of its own
// pixel; a compressing find there could overwrite another pixel's stored root
// with a non-root ancestor after that pixel's thread has written it.
__device__ __forceinline__ int uf_root(const int32_t *parent, int x) {
  int p = parent[x];
  while (p != x) {
    x = p;
    p = parent[x];
  }
  return x;
}

__global__ void k_flatten(const uint8_t *__restrict__ vcc, int N, int32_t *parent,
                          int32_t *__restrict__ size) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  size[p] = 0;
  if (!vcc[p]) return;
  parent[p] = uf_root(parent, p);
}

__global__ void k_region_stats(const uint32_t *__restrict__ F, const uint8_t *__restrict__ vcc, int W,
                               int H, int lq, const int32_t *__restrict__ parent, int32_t *size,
                               uint8_t *touch) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = p < W * H && vcc[p];
  const int root = act ? parent[p] : -1;
  // neighbouring pixels mostly share a region: one atomic per root and warp
  const unsigned grp = __match_any_sync(0xffffffffu, root);
  if (act && (__ffs(grp) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&size[root], __popc(grp));
  if (!act) return;
  const int x = p % W, y = p / W;
  const uint32_t f = F[p];
  bool t = false;
  if (x > 0 && !vcc[p - 1] && close3(f, F[p - 1], lq)) t = true;
  if (x + 1 < W && !vcc[p + 1] && close3(f, F[p + 1], lq)) t = true;
  if (y > 0 && !vcc[p - W] && close3(f, F[p - W], lq)) t = true;
  if (y + 1 < H && !vcc[p + W] && close3(f, F[p + W], lq)) t = true;
  if (t) touch[root] = 1;
}

__global__ void k_region_apply(const uint8_t *__restrict__ vcc, int N, int s,
                               const int32_t *__restrict__ parent, const int32_t *__restrict__ size,
                               const uint8_t *__restrict__ touch, uint8_t *__restrict__ valid,
                               uint8_t *__restrict__ mask) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  mask[p] = 0;
  uint8_t v = vcc[p];
  if (v) {
    const int root = parent[p];
    if (size[root] < s && touch[root]) v = 0;
  }
  valid[p] = v;
}

// Sec. 3.5 sparsification, in three parallel steps that keep the output in block
// raster order: k_blocks picks each aligned 3x3 block's survivor (>= e valid
// points, the smallest sum of the two consistency errors, raster-first on ties)
// and counts the picks of its
// CTA; k_pick_scan turns the per-CTA counts into offsets; k_pick_write writes
// every pick at its CTA's offset plus its rank inside the CTA.
constexpr int PICK_CTA = 256;

__device__ __forceinline__ int cta_exclusive_rank(bool flag, int *s_warp, int &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) s_warp[warp] = __popc(b);
  __syncthreads();
  int before = 0;
  total = 0;
  for (int w = 0; w < PICK_CTA / 32; w++) {
    if (w < warp) before += s_warp[w];
    total += s_warp[w];
  }
  return before + __popc(b & ((1u << lane) - 1));
}

// Sec. 3.5 ranks the samples of a block by the sum of their two consistency-check
// errors |F(p) + Fb_j(p + F(p))| (Eq. 5): sqrt(e1) + sqrt(e2) of the squared
// errors. sum_sqrt_lt(a, b, c, d) is sqrt(a) + sqrt(b) < sqrt(c) + sqrt(d),
// exactly, for 0 <= a..d < 2^28 (a passing pixel has e_j < eps^2 <= 10^6):
// squaring both non-negative sides gives sqrt(4ab) - sqrt(4cd) < (c+d) - (a+b);
// the left side has the sign of 4ab - 4cd, and the two undecided cases are
// squared once more, in 128-bit integers.
__device__ __forceinline__ bool sum_sqrt_lt(long long a, long long b, long long c, long long d) {
  const __int128 p = (__int128)4 * a * b, q = (__int128)4 * c * d;
  const __int128 t = (__int128)(c + d) - (__int128)(a + b);
  if (p == q) return t > 0;
  if (p < q) {  // negative left side
    if (t >= 0) return true;
    const __int128 m = q - p - t * t;  // need sqrt(q) - sqrt(p) > -t: m > -2t sqrt(p)
    return m > 0 && m * m > 4 * t * t * p;
  }
  if (t <= 0) return false;
  const __int128 m = p - q - t * t;  // need sqrt(p) - sqrt(q) < t: m < 2t sqrt(q)
  return m < 0 || m * m < 4 * t * t * q;
}

// Squared consistency errors of a pixel that passed Eq. 5 (target inside the image).
__device__ __forceinline__ void pixel_errors(const uint32_t *F, const uint32_t *Fb1,
                                             const uint32_t *Fb2, int W, int lq, int p,
                                             long long &e1, long long &e2) {
  const uint32_t f = F[p];
  int qx, qy;
  target_pixel(p % W, p / W, f, lq, qx, qy);
  const int q = qy * W + qx;
  const uint32_t b1 = Fb1[q], b2 = Fb2[q];
  const long long a0 = flow_dx(f) + flow_dx(b1), a1 = flow_dy(f) + flow_dy(b1);
  const long long c0 = flow_dx(f) + flow_dx(b2), c1 = flow_dy(f) + flow_dy(b2);
  e1 = a0 * a0 + a1 * a1;
  e2 = c0 * c0 + c1 * c1;
}

__global__ void __launch_bounds__(PICK_CTA) k_blocks(const uint8_t *__restrict__ valid,
                                                     const uint32_t *__restrict__ F,
                                                     const uint32_t *__restrict__ Fb1,
                                                     const uint32_t *__restrict__ Fb2, int W, int H,
                                                     int lq, int e, int32_t *__restrict__ pick,
                                                     int32_t *__restrict__ cta_count) {
  __shared__ int s_warp[PICK_CTA / 32];
  const int BX = (W + 2) / 3, BY = (H + 2) / 3;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  int sel = -1;
  if (b < BX * BY) {
    const int bx = b % BX, by = b / BX;
    int cnt = 0, best = -1;
    long long be1 = 0, be2 = 0;
    for (int y = 3 * by; y < min(3 * by + 3, H); y++)
      for (int x = 3 * bx; x < min(3 * bx + 3, W); x++) {
        const int p = y * W + x;
        if (!valid[p]) continue;
        cnt++;
        long long e1, e2;
        pixel_errors(F, Fb1, Fb2, W, lq, p, e1, e2);
        if (best < 0 || sum_sqrt_lt(e1, e2, be1, be2)) {
          best = p;
          be1 = e1;
          be2 = e2;
        }
      }
    sel = (cnt >= e) ? best : -1;
    pick[b] = sel;
  }
  int total;
  cta_exclusive_rank(sel >= 0, s_warp, total);
  if (threadIdx.x == 0) cta_count[blockIdx.x] = total;
}

// One CTA: exclusive scan of the per-CTA pick counts (in place) and the total.
__global__ void __launch_bounds__(1024) k_pick_scan(int32_t *__restrict__ cta_count, int n,
                                                    int32_t *__restrict__ n_sparse) {
  __shared__ int part[1024];
  const int t = threadIdx.x, per = (n + 1023) / 1024;
  const int b0 = min(t * per, n), b1 = min(b0 + per, n);
  int cnt = 0;
  for (int b = b0; b < b1; b++) cnt += cta_count[b];
  part[t] = cnt;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - cnt;
  for (int b = b0; b < b1; b++) {
    const int c = cta_count[b];
    cta_count[b] = run;
    run += c;
  }
  if (t == 1023) *n_sparse = part[1023];
}

__global__ void __launch_bounds__(PICK_CTA) k_pick_write(const int32_t *__restrict__ pick, int nb,
                                                         int W, const uint32_t *__restrict__ F,
                                                         const int32_t *__restrict__ cta_offset,
                                                         int32_t *__restrict__ sparse,
                                                         uint8_t *__restrict__ mask) {
  __shared__ int s_warp[PICK_CTA / 32];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = b < nb ? pick[b] : -1;
  int total;
  const int r = cta_exclusive_rank(p >= 0, s_warp, total);
  if (p < 0) return;
  const int out = cta_offset[blockIdx.x] + r;
  const uint32_t f = F[p];
  sparse[4 * out] = p % W;
  sparse[4 * out + 1] = p / W;
  sparse[4 * out + 2] = flow_dx(f);
  sparse[4 * out + 3] = flow_dy(f);
  mask[p] = 1;
}

size_t filter_scratch_bytes(int W, int H) {
  const size_t N = (size_t)W * H, NB = (size_t)((W + 2) / 3) * ((H + 2) / 3);
  Arena a;
  a.take<uint8_t>(N);
  a.take<int32_t>(N);
  a.take<int32_t>(N);
  a.take<uint8_t>(N);
  a.take<int32_t>(NB);
  a.take<int32_t>((NB + PICK_CTA - 1) / PICK_CTA);
  return a.off;
}

ff_status launch_filter(const uint32_t *F, const uint32_t *Fb1, const uint32_t *Fb2, int W, int H,
                        int eps, int e, int s, int q, uint8_t *valid, int32_t *err_sum,
                        int32_t *sparse, int32_t *n_sparse, uint8_t *mask, void *scratch,
                        cudaStream_t st) {
  if (q != 1 && q != 2 && q != 4) return FF_ERR_INVALID_ARG;
  const int lq = q == 4 ? 2 : q - 1;
  const int N = W * H, NB = ((W + 2) / 3) * ((H + 2) / 3);
  Arena a(scratch, (size_t)-1);
  uint8_t *vcc = a.take<uint8_t>(N);
  int32_t *parent = a.take<int32_t>(N);
  int32_t *size = a.take<int32_t>(N);
  uint8_t *touch = a.take<uint8_t>(N);
  int32_t *pick = a.take<int32_t>(NB);
  const int ncta = (NB + PICK_CTA - 1) / PICK_CTA;
  int32_t *cta_count = a.take<int32_t>(ncta);
  const int B = 256, g = (N + B - 1) / B;
  if (cudaMemsetAsync(touch, 0, N, st) != cudaSuccess) return FF_ERR_CUDA;
  k_consistency<<<g, B, 0, st>>>(F, Fb1, Fb2, W, H, eps, lq, vcc, err_sum, parent);
  FF_CHECK_LAUNCH();
  k_union<<<g, B, 0, st>>>(F, vcc, W, H, lq, parent);
  FF_CHECK_LAUNCH();
  k_flatten<<<g, B, 0, st>>>(vcc, N, parent, size);
  FF_CHECK_LAUNCH();
  k_region_stats<<<g, B, 0, st>>>(F, vcc, W, H, lq, parent, size, touch);
  FF_CHECK_LAUNCH();
  k_region_apply<<<g, B, 0, st>>>(vcc, N, s, parent, size, touch, valid, mask);
  FF_CHECK_LAUNCH();
  k_blocks<<<ncta, PICK_CTA, 0, st>>>(valid, F, Fb1, Fb2, W, H, lq, e, pick, cta_count);
  FF_CHECK_LAUNCH();
  k_pick_scan<<<1, 1024, 0, st>>>(cta_count, ncta, n_sparse);
  FF_CHECK_LAUNCH();
  k_pick_write<<<ncta, PICK_CTA, 0, st>>>(pick, NB, W, F, cta_count, sparse, mask);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

}  // namespace ff
