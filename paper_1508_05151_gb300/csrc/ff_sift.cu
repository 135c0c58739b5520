// Sec. 3.3, the second data term: SIFT flow. Dense SIFT vectors (integer), their
// exact PCA statistics, the PCA basis (float64 Jacobi rotations in one CTA), the
// quantised colours, and the kd initialisation and level search with E_d on the
// colours; the whole path for one pair on top of them.
//
// Colour layout inside the search: every pixel's S channels packed into one
// (S <= 16) or two (S <= 32) 16-byte words, zero padded, pixel major. A tap then
// costs one or two 16-byte loads per side, |a - b| per byte (vabsdiffu4) and the
// squared sum by dp4a, then an exact integer square root.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "ff_internal.cuh"

namespace ff {

constexpr int SIFT_DIM = 128;
constexpr int SIFT_CELL = 3;       // cell edge in pixels
constexpr int SIFT_SHIFT = 12;     // basis components in units of 2^-12
constexpr int SIFT_MAX_S = 30;
constexpr int SIFT_GROUP = 16;     // lanes per patch evaluation in the search (half a warp)

__constant__ int c_dir_c[8] = {256, 181, 0, -181, -256, -181, 0, 181};
__constant__ int c_dir_s[8] = {0, 181, 256, 181, 0, -181, -256, -181};

// ----------------------------------------------------------- integer roots ---
// floor(sqrt(x)) for x < 2^46: a float estimate (within 1 of the root there),
// then exact integer corrections.
__device__ __forceinline__ uint64_t isqrt_u64(uint64_t x) {
  uint64_t s = (uint64_t)sqrtf((float)x);
  for (int it = 0; it < 4 && s * s > x; it++) s--;
  for (int it = 0; it < 4 && (s + 1) * (s + 1) <= x; it++) s++;
  return s;
}
__device__ __forceinline__ uint32_t isqrt_u32(uint32_t x) {  // x < 2^30
  uint32_t s = (uint32_t)sqrtf((float)x);
  for (int it = 0; it < 2 && s * s > x; it++) s--;
  for (int it = 0; it < 2 && (s + 1) * (s + 1) <= x; it++) s++;
  return s;
}
// floor(num / den) for num / den < 2^20 and num < 2^62: a float estimate, then
// exact corrections.
__device__ __forceinline__ uint64_t udiv_small(uint64_t num, uint64_t den) {
  uint64_t y = (uint64_t)((float)num * __frcp_rn((float)den));
  for (int it = 0; it < 4 && y * den > num; it++) y--;
  for (int it = 0; it < 4 && (y + 1) * den <= num; it++) y++;
  return y;
}
__host__ __device__ __forceinline__ long long floor_div_ll(long long a, long long b) {
  long long q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// ------------------------------------------------------------- descriptor ----
// One CTA per 16 x 16 output tile. The orientation responses of the tile's
// window (offsets -2c .. 16 + 2c - 1, clamped) go to shared memory, then the
// row sums over c pixels; each thread sums its pixel's 128 cells from those,
// three times (norm, clipped norm, quantised values).
constexpr int SD_T = 16;
constexpr int SD_E = SD_T + 4 * SIFT_CELL;   // 28
constexpr int SD_RW = SD_T + 3 * SIFT_CELL;  // 25

__device__ __forceinline__ int grey_at(const uint8_t *img, int W, int H, int x, int y) {
  const uint8_t *p = img + 3 * ((size_t)clampi(y, 0, H - 1) * W + clampi(x, 0, W - 1));
  return p[0] + p[1] + p[2];
}

__global__ void __launch_bounds__(256) k_sift_desc(const uint8_t *img, int W, int H,
                                                   uint8_t *desc) {
  __shared__ int32_t so[8][SD_E][SD_E];
  __shared__ int32_t rb[8][SD_E][SD_RW];
  const int x0 = blockIdx.x * SD_T, y0 = blockIdx.y * SD_T, tid = threadIdx.x;
  for (int i = tid; i < SD_E * SD_E; i += blockDim.x) {
    const int v = i / SD_E, u = i % SD_E;
    const int x = clampi(x0 - 2 * SIFT_CELL + u, 0, W - 1);
    const int y = clampi(y0 - 2 * SIFT_CELL + v, 0, H - 1);
    const int gx = grey_at(img, W, H, x + 1, y) - grey_at(img, W, H, x - 1, y);
    const int gy = grey_at(img, W, H, x, y + 1) - grey_at(img, W, H, x, y - 1);
#pragma unroll
    for (int k = 0; k < 8; k++) so[k][v][u] = max(0, gx * c_dir_c[k] + gy * c_dir_s[k]);
  }
  __syncthreads();
  for (int i = tid; i < 8 * SD_E * SD_RW; i += blockDim.x) {
    const int k = i / (SD_E * SD_RW), rem = i % (SD_E * SD_RW), v = rem / SD_RW, j = rem % SD_RW;
    int acc = 0;
#pragma unroll
    for (int d = 0; d < SIFT_CELL; d++) acc += so[k][v][j + d];
    rb[k][v][j] = acc;
  }
  __syncthreads();
  const int tx = tid & (SD_T - 1), ty = tid / SD_T, px = x0 + tx, py = y0 + ty;
  if (px >= W || py >= H) return;
  auto cell = [&](int d) -> uint32_t {
    const int k = d & 7, i = (d >> 3) & 3, j = d >> 5;
    int acc = 0;
#pragma unroll
    for (int e = 0; e < SIFT_CELL; e++) acc += rb[k][ty + SIFT_CELL * j + e][tx + SIFT_CELL * i];
    return (uint32_t)acc;
  };
  uint64_t N2 = 0;
  for (int d = 0; d < SIFT_DIM; d++) {
    const uint64_t h = cell(d);
    N2 += h * h;
  }
  const uint64_t t = isqrt_u64(N2 / 25);
  uint64_t M2 = 0;
  for (int d = 0; d < SIFT_DIM; d++) {
    const uint64_t h = min((uint64_t)cell(d), t);
    M2 += h * h;
  }
  uint4 *out = (uint4 *)(desc + ((size_t)py * W + px) * SIFT_DIM);
  for (int w16 = 0; w16 < SIFT_DIM / 16; w16++) {
    uint32_t wv[4];
#pragma unroll
    for (int w = 0; w < 4; w++) {
      uint32_t word = 0;
#pragma unroll
      for (int b = 0; b < 4; b++) {
        const int d = w16 * 16 + w * 4 + b;
        uint32_t q = 0;
        if (M2 > 0) {
          const uint64_t h = min((uint64_t)cell(d), t);
          q = min(255u, isqrt_u32((uint32_t)udiv_small((h * h) << 18, M2)));
        }
        word |= q << (8 * b);
      }
      wv[w] = word;
    }
    out[w16] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  }
}

// ---------------------------------------------------------------- moments ----
// Each CTA takes MOM_CHUNK descriptors, staged MOM_STAGE at a time in shared
// memory transposed to [dimension][pixel] bytes; thread (ti, tj) accumulates the
// 8 x 8 block (8 ti + a, 8 tj + b) of the Gram matrix with dp4a over 4 pixels per
// word (exact in 32 bits: MOM_CHUNK * 255^2 < 2^32), then adds it to the 64-bit
// totals.
constexpr int MOM_CHUNK = 4096, MOM_STAGE = 64, MOM_PITCH = MOM_STAGE + 4;

__global__ void __launch_bounds__(256) k_sift_moments(const uint8_t *desc, int N,
                                                      unsigned long long *sum,
                                                      unsigned long long *gram) {
  __shared__ __align__(16) uint8_t tile[SIFT_DIM * MOM_PITCH];
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  uint32_t acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; a++)
#pragma unroll
    for (int b = 0; b < 8; b++) acc[a][b] = 0;
  uint32_t sacc = 0;
  const long long p_begin = (long long)blockIdx.x * MOM_CHUNK;
  const long long p_end = min((long long)N, p_begin + MOM_CHUNK);
  for (long long p0 = p_begin; p0 < p_end; p0 += MOM_STAGE) {
    {
      const int pl = tid >> 2, part = tid & 3;
      const long long p = p0 + pl;
      uint4 a = make_uint4(0, 0, 0, 0), b = a;
      if (p < p_end) {
        const uint4 *src = (const uint4 *)(desc + (size_t)p * SIFT_DIM + 32 * part);
        a = src[0];
        b = src[1];
      }
      const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 32; i++)
        tile[(32 * part + i) * MOM_PITCH + pl] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
    }
    __syncthreads();
    const uint32_t *tw = (const uint32_t *)tile;
#pragma unroll 2
    for (int w = 0; w < MOM_STAGE / 4; w++) {
      uint32_t ra[8], rv[8];
#pragma unroll
      for (int a = 0; a < 8; a++) ra[a] = tw[(8 * ti + a) * (MOM_PITCH / 4) + w];
#pragma unroll
      for (int b = 0; b < 8; b++) rv[b] = tw[(8 * tj + b) * (MOM_PITCH / 4) + w];
#pragma unroll
      for (int a = 0; a < 8; a++)
#pragma unroll
        for (int b = 0; b < 8; b++) acc[a][b] = __dp4a(ra[a], rv[b], acc[a][b]);
      if (tid < SIFT_DIM) sacc = __dp4a(tw[tid * (MOM_PITCH / 4) + w], 0x01010101u, sacc);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 8; a++)
#pragma unroll
    for (int b = 0; b < 8; b++)
      if (acc[a][b]) atomicAdd(&gram[(8 * ti + a) * SIFT_DIM + 8 * tj + b], (unsigned long long)acc[a][b]);
  if (tid < SIFT_DIM && sacc) atomicAdd(&sum[tid], (unsigned long long)sacc);
}

// -------------------------------------------------------------------- PCA ----
// One CTA: the covariance in shared memory (128 x 128 float64), cyclic Jacobi
// rotations in round-robin order (64 disjoint pairs per round, 127 rounds per
// sweep: index 127 fixed, the others rotating), the eigenvectors accumulated as
// the rows of VT in global memory. Sweeps stop once the off-diagonal squares sum
// to at most 1e-30 of the diagonal's, at most PCA_MAX_SWEEPS.
constexpr int PCA_THREADS = 1024;
constexpr int PCA_MAX_SWEEPS = 40;
constexpr size_t PCA_SMEM = sizeof(double) * SIFT_DIM * SIFT_DIM;

__device__ double block_sum_pca(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
  return t;
}

__global__ void __launch_bounds__(PCA_THREADS) k_sift_pca(const unsigned long long *sum,
                                                          const unsigned long long *gram,
                                                          long long count, int S, double *VT,
                                                          int16_t *basis, int32_t *offset,
                                                          double *eigval, DeviceStatus *status) {
  extern __shared__ double A[];  // [128][128]
  __shared__ double rc[64], rs[64], red[PCA_THREADS / 32];
  __shared__ int rp[64], rq[64], rank_of[SIFT_DIM];
  const int tid = threadIdx.x;
  const double inv = 1.0 / (double)count;
  for (int i = tid; i < SIFT_DIM * SIFT_DIM; i += blockDim.x) {
    const int a = i >> 7, b = i & 127;
    const double ma = (double)sum[a] * inv, mb = (double)sum[b] * inv;
    A[i] = (double)gram[i] * inv - ma * mb;
    VT[i] = a == b ? 1.0 : 0.0;
  }
  __syncthreads();
  bool converged = false;
  for (int sweep = 0; sweep < PCA_MAX_SWEEPS; sweep++) {
    double off = 0, dia = 0;
    for (int i = tid; i < SIFT_DIM * SIFT_DIM; i += blockDim.x) {
      const double v = A[i];
      if ((i >> 7) == (i & 127)) dia += v * v;
      else off += v * v;
    }
    off = block_sum_pca(off, red);
    dia = block_sum_pca(dia, red);
    if (off <= 1e-30 * dia) {
      converged = true;
      break;
    }
    for (int m = 0; m < SIFT_DIM - 1; m++) {
      if (tid < 64) {
        int p = tid == 0 ? m : (m + tid) % 127, q = tid == 0 ? 127 : (m - tid + 127) % 127;
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const double apq = A[p * SIFT_DIM + q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double theta = (A[q * SIFT_DIM + q] - A[p * SIFT_DIM + p]) / (2.0 * apq);
          const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
        }
        rc[tid] = c;
        rs[tid] = s;
        rp[tid] = p;
        rq[tid] = q;
      }
      __syncthreads();
      // A <- J^T A (rows p, q), VT <- J^T VT (the same rows of VT = V^T)
      for (int i = tid; i < 64 * SIFT_DIM; i += blockDim.x) {
        const int k = i >> 7, j = i & 127, p = rp[k], q = rq[k];
        const double c = rc[k], s = rs[k];
        const double ap = A[p * SIFT_DIM + j], aq = A[q * SIFT_DIM + j];
        A[p * SIFT_DIM + j] = c * ap - s * aq;
        A[q * SIFT_DIM + j] = s * ap + c * aq;
        const double vp = VT[p * SIFT_DIM + j], vq = VT[q * SIFT_DIM + j];
        VT[p * SIFT_DIM + j] = c * vp - s * vq;
        VT[q * SIFT_DIM + j] = s * vp + c * vq;
      }
      __syncthreads();
      // A <- A J (columns p, q); lanes of a warp take different pairs of one row
      for (int i = tid; i < 64 * SIFT_DIM; i += blockDim.x) {
        const int j = i >> 6, k = i & 63, p = rp[k], q = rq[k];
        const double c = rc[k], s = rs[k];
        const double ap = A[j * SIFT_DIM + p], aq = A[j * SIFT_DIM + q];
        A[j * SIFT_DIM + p] = c * ap - s * aq;
        A[j * SIFT_DIM + q] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
  if (!converged && tid == 0) raise_status(status, DEV_ERR_TIMEOUT, -1, PCA_MAX_SWEEPS);
  // ranks: descending eigenvalue, ties to the lower index
  if (tid < SIFT_DIM) {
    const double lam = A[tid * (SIFT_DIM + 1)];
    int rank = 0;
    for (int j = 0; j < SIFT_DIM; j++) {
      const double lj = A[j * (SIFT_DIM + 1)];
      rank += (lj > lam) || (lj == lam && j < tid);
    }
    rank_of[rank] = tid;
    if (eigval) eigval[rank] = lam;
  }
  __syncthreads();
  const double gain = 127.0 / (3.0 * sqrt(fmax(A[rank_of[0] * (SIFT_DIM + 1)], 1.0)));
  const int warp = tid >> 5, lane = tid & 31;
  for (int s = warp; s < S; s += blockDim.x >> 5) {
    const double *v = VT + (size_t)rank_of[s] * SIFT_DIM;
    double best = -1.0;
    int bidx = SIFT_DIM;
    for (int i = lane; i < SIFT_DIM; i += 32) {
      const double a = fabs(v[i]);
      if (a > best) {
        best = a;
        bidx = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) {
        best = ob;
        bidx = oi;
      }
    }
    const double sg = v[bidx] < 0.0 ? -1.0 : 1.0;
    long long num = 0;
    for (int i = lane; i < SIFT_DIM; i += 32) {
      const double x = floor((double)(1 << SIFT_SHIFT) * gain * (sg * v[i]) + 0.5);
      const int b = (int)fmin(fmax(x, -32767.0), 32767.0);
      basis[s * SIFT_DIM + i] = (int16_t)b;
      num += (long long)b * (long long)sum[i];
    }
    for (int o = 16; o > 0; o >>= 1) num += __shfl_xor_sync(0xffffffffu, num, o);
    if (lane == 0) offset[s] = (int32_t)(2048 - floor_div_ll(2 * num + count, 2 * count));
  }
}

// ---------------------------------------------------------------- colours ----
__global__ void __launch_bounds__(256) k_sift_colors(const uint8_t *desc, int N,
                                                     const int16_t *basis,
                                                     const int32_t *offset, int S,
                                                     uint8_t *col) {
  __shared__ int32_t sB[SIFT_MAX_S][SIFT_DIM];
  __shared__ int32_t so[SIFT_MAX_S];
  for (int i = threadIdx.x; i < S * SIFT_DIM; i += blockDim.x) sB[i / SIFT_DIM][i % SIFT_DIM] = basis[i];
  if (threadIdx.x < S) so[threadIdx.x] = offset[threadIdx.x];
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  uint32_t w[32];
  const uint4 *src = (const uint4 *)(desc + (size_t)p * SIFT_DIM);
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const uint4 v = src[i];
    w[4 * i] = v.x;
    w[4 * i + 1] = v.y;
    w[4 * i + 2] = v.z;
    w[4 * i + 3] = v.w;
  }
  for (int s = 0; s < S; s++) {
    int acc = 0;  // |sum| <= 32767 * 255 * 128 < 2^31
#pragma unroll
    for (int i = 0; i < SIFT_DIM; i++) acc += sB[s][i] * (int)((w[i >> 2] >> (8 * (i & 3))) & 0xffu);
    const long long v = 128 + floor_div_ll((long long)acc + so[s], 1ll << SIFT_SHIFT);
    col[(size_t)(s / 3) * N * 3 + (size_t)p * 3 + s % 3] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
  }
}

// Level-n colour groups -> one or two zero-padded 16-byte words per pixel.
__global__ void __launch_bounds__(256) k_sift_pack(const uint8_t *col, int N, int S, int nw4,
                                                   uint4 *K) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int s = 0; s < S; s++)
    w[s >> 2] |= (uint32_t)col[(size_t)(s / 3) * N * 3 + (size_t)p * 3 + s % 3] << (8 * (s & 3));
  K[(size_t)p * nw4] = make_uint4(w[0], w[1], w[2], w[3]);
  if (nw4 == 2) K[(size_t)p * nw4 + 1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// ----------------------------------------------------------------- search ----
struct SiftLevel {
  const uint4 *Ks, *Kt;  // packed level-n colours of the source and target frame
  int W, H, n, Gx, Gy, flow_id;
  const uint32_t *flow_coarse;  // level-2n flows or nullptr
  int Gxc;
  unsigned long long *evals;    // evaluation counters of the pass kernel or nullptr
};

// Squared colour distance of one tap from its loaded words, then the fixed-point
// norm.
template <int NW4>
__device__ __forceinline__ int sift_tap_words(const uint4 *a, const uint4 *b) {
  uint32_t acc = 0;
#pragma unroll
  for (int w = 0; w < NW4; w++) {
    uint32_t d = __vabsdiffu4(a[w].x, b[w].x);
    acc = __dp4a(d, d, acc);
    d = __vabsdiffu4(a[w].y, b[w].y);
    acc = __dp4a(d, d, acc);
    d = __vabsdiffu4(a[w].z, b[w].z);
    acc = __dp4a(d, d, acc);
    d = __vabsdiffu4(a[w].w, b[w].w);
    acc = __dp4a(d, d, acc);
  }
  return (int)isqrt_u32(acc << 8);  // acc <= 30 * 255^2
}

// E_d of source pixel (px, py) against up to two targets (X0, Y0), (X1, Y1) at
// once: a group of 16 lanes (mask gmask) splits the (2R+1)^2 taps, tap
// t = lane + 16 k; the source word of a tap is loaded once for both targets. Sums
// are complete in every lane; a target with use* false gets no defined cost.
// use0 / use1 are uniform over the group.
template <int R, int NW4, bool TWO>
__device__ __forceinline__ void sift_costs(const SiftLevel &L, int px, int py, int X0, int Y0,
                                           bool use0, int X1, int Y1, bool use1, int lg,
                                           unsigned gmask, int &e0, int &e1) {
  constexpr int D = 2 * R + 1, DD = D * D, KT = (DD + SIFT_GROUP - 1) / SIFT_GROUP;
  int a0 = 0, a1 = 0;
#pragma unroll 4
  for (int k = 0; k < KT; k++) {
    const int t = lg + SIFT_GROUP * k;
    if (t < DD) {
      const int v = t / D - R, u = t % D - R;
      const int xs = clampi(px + L.n * u, 0, L.W - 1), ys = clampi(py + L.n * v, 0, L.H - 1);
      uint4 sv[NW4], tv[NW4];
      const uint4 *src = L.Ks + ((size_t)ys * L.W + xs) * NW4;
#pragma unroll
      for (int w = 0; w < NW4; w++) sv[w] = __ldg(src + w);
      if (use0) {
        const int xt = clampi(X0 + L.n * u, 0, L.W - 1), yt = clampi(Y0 + L.n * v, 0, L.H - 1);
        const uint4 *g = L.Kt + ((size_t)yt * L.W + xt) * NW4;
#pragma unroll
        for (int w = 0; w < NW4; w++) tv[w] = __ldg(g + w);
        a0 += sift_tap_words<NW4>(sv, tv);
      }
      if (TWO && use1) {
        const int xt = clampi(X1 + L.n * u, 0, L.W - 1), yt = clampi(Y1 + L.n * v, 0, L.H - 1);
        const uint4 *g = L.Kt + ((size_t)yt * L.W + xt) * NW4;
#pragma unroll
        for (int w = 0; w < NW4; w++) tv[w] = __ldg(g + w);
        a1 += sift_tap_words<NW4>(sv, tv);
      }
    }
  }
#pragma unroll
  for (int o = SIFT_GROUP / 2; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(gmask, a0, o);
    if (TWO) a1 += __shfl_xor_sync(gmask, a1, o);
  }
  e0 = a0;
  e1 = a1;
}

template <int R, int NW4>
__device__ __forceinline__ int sift_cost(const SiftLevel &L, int px, int py, int X, int Y, int lg,
                                         unsigned gmask) {
  int e0, e1;
  sift_costs<R, NW4, false>(L, px, py, X, Y, true, X, Y, false, lg, gmask, e0, e1);
  return e0;
}

template <int R, int NW4>
__device__ __forceinline__ void sift_cost2(const SiftLevel &L, int px, int py, int X0, int Y0,
                                           bool use0, int X1, int Y1, bool use1, int lg,
                                           unsigned gmask, int &e0, int &e1) {
  sift_costs<R, NW4, true>(L, px, py, X0, Y0, use0, X1, Y1, use1, lg, gmask, e0, e1);
}

struct SiftKdQuery {
  const int32_t *perm, *split_dim, *split_val;
  int N, D;
  const int32_t *qfeat;  // [G][28] WHT features of the source frame at the grid points
  uint32_t *flow;
  int32_t *cost;
  DeviceStatus *status;
};

// Eq. 1 / Eq. 4 with the SIFT flow data term: descend the tree with the grid
// point's WHT vector, rerank the leaf by E_d (ties to the lower pixel index).
template <int R, int NW4>
__global__ void __launch_bounds__(256) k_sift_kd_query(SiftLevel L, SiftKdQuery Q) {
  const int G = L.Gx * L.Gy;
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) / SIFT_GROUP;
  const int lg = threadIdx.x & (SIFT_GROUP - 1);
  const unsigned gmask = 0xffffu << (threadIdx.x & 16);
  if (g >= G) return;  // uniform per group
  const int px = (g % L.Gx) * L.n, py = (g / L.Gx) * L.n;
  int leaf = 0;
  if (lg == 0) {
    const int32_t *q = Q.qfeat + (size_t)g * FEAT_STRIDE;
    int node = 0;
    for (int d = 0; d < Q.D; d++) {
      int sd = Q.split_dim[node];
      if ((unsigned)sd >= (unsigned)NFEAT) {
        raise_status(Q.status, DEV_ERR_BOUNDS, g, node);
        sd = 0;
      }
      node = (q[sd] < Q.split_val[node]) ? 2 * node + 1 : 2 * node + 2;
    }
    leaf = node - ((1 << Q.D) - 1);
  }
  leaf = __shfl_sync(gmask, leaf, threadIdx.x & 16);
  const int b = seg_begin(Q.N, Q.D, leaf), e = seg_begin(Q.N, Q.D, leaf + 1);
  int best = COST_UNSET, bidx = 0x7fffffff;
  for (int c = b; c < e; c += 2) {
    int idx[2] = {Q.perm[c], c + 1 < e ? Q.perm[c + 1] : -1};
    bool use[2];
    for (int i = 0; i < 2; i++) {
      use[i] = (unsigned)idx[i] < (unsigned)Q.N;  // uniform over the group
      if (!use[i] && (i == 0 || c + 1 < e) && lg == 0) raise_status(Q.status, DEV_ERR_BOUNDS, g, c + i);
    }
    int cost[2];
    sift_cost2<R, NW4>(L, px, py, use[0] ? idx[0] % L.W : 0, use[0] ? idx[0] / L.W : 0, use[0],
                       use[1] ? idx[1] % L.W : 0, use[1] ? idx[1] / L.W : 0, use[1], lg, gmask,
                       cost[0], cost[1]);
    for (int i = 0; i < 2; i++)
      if (use[i] && (cost[i] < best || (cost[i] == best && idx[i] < bidx))) {
        best = cost[i];
        bidx = idx[i];
      }
  }
  if (lg == 0) {
    Q.flow[g] = pack_flow(bidx % L.W - px, bidx / L.W - py);
    Q.cost[g] = best;
  }
}

// Sec. 3.2 level transition: grid points with both coordinates even take the
// coarser level's flow (cost re-evaluated), all others start without a flow.
template <int R, int NW4>
__global__ void __launch_bounds__(256) k_sift_seed(SiftLevel L, uint32_t *flow, int32_t *cost) {
  const int G = L.Gx * L.Gy;
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) / SIFT_GROUP;
  const int lg = threadIdx.x & (SIFT_GROUP - 1);
  const unsigned gmask = 0xffffu << (threadIdx.x & 16);
  if (g >= G) return;
  const int gx = g % L.Gx, gy = g / L.Gx, px = gx * L.n, py = gy * L.n;
  uint32_t f = 0;
  int c = COST_UNSET;
  if (!(gx & 1) && !(gy & 1)) {
    const uint32_t fc = L.flow_coarse[(size_t)(gy >> 1) * L.Gxc + (gx >> 1)];
    const int X = clampi(px + flow_dx(fc), 0, L.W - 1), Y = clampi(py + flow_dy(fc), 0, L.H - 1);
    c = sift_cost<R, NW4>(L, px, py, X, Y, lg, gmask);
    f = pack_flow(X - px, Y - py);
  }
  if (lg == 0) {
    flow[g] = f;
    cost[g] = c;
  }
}

// Random search step (Sec. 3.1): F + O_rnd, kept if E_d decreases; in place.
template <int R, int NW4>
__global__ void __launch_bounds__(256) k_sift_rs(SiftLevel L, uint32_t *flow, int32_t *cost,
                                                 int step, int level, int Rn, uint64_t seed) {
  const int G = L.Gx * L.Gy;
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) / SIFT_GROUP;
  const int lg = threadIdx.x & (SIFT_GROUP - 1);
  const unsigned gmask = 0xffffu << (threadIdx.x & 16);
  if (g >= G) return;
  const int c = cost[g];
  if (c == COST_UNSET) return;  // uniform per group
  const uint32_t f = flow[g];
  const int gx = g % L.Gx, gy = g / L.Gx, px = gx * L.n, py = gy * L.n;
  int dx, dy;
  rs_offset(seed, L.flow_id, level, step, gx, gy, Rn, dx, dy);
  const int X = clampi(px + flow_dx(f) + dx, 0, L.W - 1);
  const int Y = clampi(py + flow_dy(f) + dy, 0, L.H - 1);
  const int e = sift_cost<R, NW4>(L, px, py, X, Y, lg, gmask);
  if (e < c && lg == 0) {
    flow[g] = pack_flow(X - px, Y - py);
    cost[g] = e;
  }
}

// Incremental costs. A propagation candidate repeats the flow f of a neighbour q
// one grid step away (q = p + sd n along x or y). When p + f needs no clamping, the
// candidate's flow is f itself, and since every tap is clamped in absolute
// coordinates, E_d(p, f) = E_d(q, f) minus the patch column (or row) that q covers
// and p does not, plus the one p covers and q does not: offsets sd (R + 1) and
// -sd R. That is 2 (2R+1) taps instead of (2R+1)^2, exact in integers.
//
// Tap t of a candidate's list: the whole patch (mode 0), or the leaving (sign -1,
// t < 2R+1) and entering (sign +1) line of a horizontal (mode 1) or vertical
// (mode 2) source at offset sd.
template <int R>
__device__ __forceinline__ void pass_tap(int mode, int sd, int t, int &u, int &v, int &sign) {
  constexpr int D = 2 * R + 1;
  if (mode == 0) {
    u = t % D - R;
    v = t / D - R;
    sign = 1;
    return;
  }
  const bool enter = t >= D;
  const int k = (enter ? t - D : t) - R, edge = enter ? -sd * R : sd * (R + 1);
  sign = enter ? 1 : -1;
  u = mode == 1 ? edge : k;
  v = mode == 1 ? k : edge;
}

// The tap sums of both candidates of a pass (ntap[c] taps of mode[c]; 0 for an
// unused candidate), split over the 16 lanes of a group, one round of 16 taps at a
// time with both candidates' gathers issued before use. Complete in every lane.
template <int R, int NW4>
__device__ __forceinline__ void sift_pass_sums(const SiftLevel &L, int px, int py, const int *X,
                                               const int *Y, const int *ntap, const int *mode,
                                               const int *sd, int lg, unsigned gmask,
                                               int *sum) {
  int acc[2] = {0, 0};
  const int tmax = max(ntap[0], ntap[1]);
#pragma unroll 2
  for (int t0 = 0; t0 < tmax; t0 += SIFT_GROUP) {
    const int t = t0 + lg;
    uint4 sv[2][NW4], tv[2][NW4];
    int sg[2];
    bool ok[2];
#pragma unroll
    for (int c = 0; c < 2; c++) {
      ok[c] = t < ntap[c];
      int u, v;
      pass_tap<R>(mode[c], sd[c], ok[c] ? t : 0, u, v, sg[c]);
      if (ok[c]) {
        const int xs = clampi(px + L.n * u, 0, L.W - 1), ys = clampi(py + L.n * v, 0, L.H - 1);
        const int xt = clampi(X[c] + L.n * u, 0, L.W - 1), yt = clampi(Y[c] + L.n * v, 0, L.H - 1);
        const uint4 *a = L.Ks + ((size_t)ys * L.W + xs) * NW4;
        const uint4 *b = L.Kt + ((size_t)yt * L.W + xt) * NW4;
#pragma unroll
        for (int w = 0; w < NW4; w++) {
          sv[c][w] = __ldg(a + w);
          tv[c][w] = __ldg(b + w);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 2; c++)
      if (ok[c]) acc[c] += sg[c] * sift_tap_words<NW4>(sv[c], tv[c]);
  }
#pragma unroll
  for (int o = SIFT_GROUP / 2; o > 0; o >>= 1) {
    acc[0] += __shfl_xor_sync(gmask, acc[0], o);
    acc[1] += __shfl_xor_sync(gmask, acc[1], o);
  }
  sum[0] = acc[0];
  sum[1] = acc[1];
}

// Sources of pass s (Fig. 3c reading): horizontal (dx, 0) and vertical (0, dy).
__constant__ int c_pass_src[4][2] = {{-1, -1}, {1, 1}, {1, -1}, {-1, 1}};

// One propagation pass (Eq. 2) in the tiled schedule: one CTA per T x T tile
// (origin shifted by T/2 in odd passes), the tile's state in shared memory, its
// grid points in anti-diagonal wavefronts along the scan direction (each point's
// two sources lie on the previous diagonal, so this equals the sequential scan),
// one 16-lane group per point of a diagonal, both candidates costed together and
// incrementally where the neighbour's flow needs no clamping. Sources outside the
// tile are read from the start-of-pass state (fin, cin); results go to
// (fout, cout).
template <int R, int NW4>
__global__ void __launch_bounds__(SIFT_GROUP * MAX_TILE) k_sift_pass(SiftLevel L, const uint32_t *fin,
                                                   const int32_t *cin, uint32_t *fout,
                                                   int32_t *cout, int s, int T) {
  __shared__ uint32_t sf[MAX_TILE * MAX_TILE];
  __shared__ int32_t sc[MAX_TILE * MAX_TILE];
  __shared__ unsigned s_inc, s_full;
  if (threadIdx.x == 0) s_inc = s_full = 0;
  const int off = (s & 1) * (T / 2);
  const int ntx = (L.Gx + off + T - 1) / T;
  const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
  const int x0 = max(tx * T - off, 0), x1 = min(tx * T - off + T, L.Gx);
  const int y0 = max(ty * T - off, 0), y1 = min(ty * T - off + T, L.Gy);
  const int tw = x1 - x0, th = y1 - y0;
  for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
    const int lx = i % tw, ly = i / tw;
    const size_t g = (size_t)(y0 + ly) * L.Gx + x0 + lx;
    sf[ly * T + lx] = fin[g];
    sc[ly * T + lx] = cin[g];
  }
  __syncthreads();
  const int sx = c_pass_src[s][0], sy = c_pass_src[s][1];
  const int gi = threadIdx.x / SIFT_GROUP, lg = threadIdx.x & (SIFT_GROUP - 1);
  const unsigned gmask = 0xffffu << (threadIdx.x & 16);
  for (int d = 0; d < tw + th - 1; d++) {
    const int iy = gi, ix = d - gi;
    if (iy < th && ix >= 0 && ix < tw) {  // uniform per group
      const int gx = sx < 0 ? x0 + ix : x1 - 1 - ix, gy = sy < 0 ? y0 + iy : y1 - 1 - iy;
      const int px = gx * L.n, py = gy * L.n;
      const int li = (gy - y0) * T + (gx - x0);
      uint32_t f = sf[li];
      int c = sc[li];
      // candidates in order: the horizontal source, then the vertical one
      bool use[2];
      int X[2], Y[2], base[2], ntap[2], mode[2];
      const int sd[2] = {sx, sy};
#pragma unroll
      for (int cand = 0; cand < 2; cand++) {
        const int qx = gx + (cand == 0 ? sx : 0), qy = gy + (cand == 0 ? 0 : sy);
        use[cand] = qx >= 0 && qx < L.Gx && qy >= 0 && qy < L.Gy;
        X[cand] = Y[cand] = base[cand] = ntap[cand] = mode[cand] = 0;
        if (use[cand]) {
          const bool inside = qx >= x0 && qx < x1 && qy >= y0 && qy < y1;
          const size_t qg = (size_t)qy * L.Gx + qx;
          const uint32_t fq = inside ? sf[(qy - y0) * T + (qx - x0)] : fin[qg];
          const int cq = inside ? sc[(qy - y0) * T + (qx - x0)] : cin[qg];
          use[cand] = cq != COST_UNSET;
          const int xu = px + flow_dx(fq), yu = py + flow_dy(fq);
          X[cand] = clampi(xu, 0, L.W - 1);
          Y[cand] = clampi(yu, 0, L.H - 1);
          if (use[cand]) {
            const bool inc = X[cand] == xu && Y[cand] == yu;  // the neighbour's flow unchanged
            mode[cand] = inc ? 1 + cand : 0;
            base[cand] = inc ? cq : 0;
            ntap[cand] = inc ? 2 * (2 * R + 1) : (2 * R + 1) * (2 * R + 1);
          }
        }
      }
      int e[2];
      sift_pass_sums<R, NW4>(L, px, py, X, Y, ntap, mode, sd, lg, gmask, e);
      e[0] += base[0];
      e[1] += base[1];
      if (L.evals && lg == 0) {
        atomicAdd(&s_inc, (unsigned)(mode[0] != 0) + (unsigned)(mode[1] != 0));
        atomicAdd(&s_full, (unsigned)(use[0] && mode[0] == 0) + (unsigned)(use[1] && mode[1] == 0));
      }
#pragma unroll
      for (int cand = 0; cand < 2; cand++)
        if (use[cand] && e[cand] < c) {
          c = e[cand];
          f = pack_flow(X[cand] - px, Y[cand] - py);
        }
      if (lg == 0) {
        sf[li] = f;
        sc[li] = c;
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
    const int lx = i % tw, ly = i / tw;
    const size_t g = (size_t)(y0 + ly) * L.Gx + x0 + lx;
    fout[g] = sf[ly * T + lx];
    cout[g] = sc[ly * T + lx];
  }
  // incremental (kind 1) and full (kind 3) evaluations, targets gathered from the
  // colour array
  if (L.evals && threadIdx.x == 0) {
    if (s_inc) atomicAdd(L.evals + 1, (unsigned long long)s_inc);
    if (s_full) atomicAdd(L.evals + 3, (unsigned long long)s_full);
  }
}

// ------------------------------------------------------------ launchers ------
#define FF_DISPATCH_SIFT(r, nw4, KERNEL, GRID, BLOCK, SMEM, ST, ...)                    \
  do {                                                                                 \
    FF_DISPATCH_R(r, {                                                                 \
      if ((nw4) == 1) KERNEL<RR, 1><<<GRID, BLOCK, SMEM, ST>>>(__VA_ARGS__);            \
      else KERNEL<RR, 2><<<GRID, BLOCK, SMEM, ST>>>(__VA_ARGS__);                       \
    });                                                                                \
    FF_CHECK_LAUNCH();                                                                 \
  } while (0)

static int sift_nw4(int S) { return S <= 16 ? 1 : 2; }
static bool sift_S_ok(int S) { return S >= 3 && S <= SIFT_MAX_S && S % 3 == 0; }
static int grid_blocks(long long threads) { return (int)((threads + 255) / 256); }

ff_status launch_sift_descriptors(const uint8_t *img, int W, int H, uint8_t *desc, cudaStream_t st) {
  dim3 grid((W + SD_T - 1) / SD_T, (H + SD_T - 1) / SD_T);
  k_sift_desc<<<grid, 256, 0, st>>>(img, W, H, desc);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

ff_status launch_sift_moments(const uint8_t *desc, int N, unsigned long long *sum,
                              unsigned long long *gram, cudaStream_t st) {
  if (N <= 0) return FF_OK;
  k_sift_moments<<<(N + MOM_CHUNK - 1) / MOM_CHUNK, 256, 0, st>>>(desc, N, sum, gram);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

ff_status launch_sift_pca(const unsigned long long *sum, const unsigned long long *gram,
                          long long count, int S, double *VT, int16_t *basis, int32_t *offset,
                          double *eigval, DeviceStatus *status, cudaStream_t st) {
  FF_TRY(smem_opt_in((const void *)k_sift_pca, PCA_SMEM));
  k_sift_pca<<<1, PCA_THREADS, PCA_SMEM, st>>>(sum, gram, count, S, VT, basis, offset, eigval,
                                              status);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

ff_status launch_sift_colors(const uint8_t *desc, int N, const int16_t *basis,
                             const int32_t *offset, int S, uint8_t *col, cudaStream_t st) {
  k_sift_colors<<<grid_blocks(N), 256, 0, st>>>(desc, N, basis, offset, S, col);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

ff_status launch_sift_pack(const uint8_t *col, int N, int S, uint4 *K, cudaStream_t st) {
  k_sift_pack<<<grid_blocks(N), 256, 0, st>>>(col, N, S, sift_nw4(S), K);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

static SiftLevel make_sift_level(const uint4 *Ks, const uint4 *Kt, int W, int H, int n,
                                 int flow_id, const uint32_t *flow_coarse) {
  SiftLevel L;
  L.Ks = Ks;
  L.Kt = Kt;
  L.W = W;
  L.H = H;
  L.n = n;
  L.Gx = (W + n - 1) / n;
  L.Gy = (H + n - 1) / n;
  L.flow_id = flow_id;
  L.flow_coarse = flow_coarse;
  L.Gxc = (W + 2 * n - 1) / (2 * n);
  L.evals = nullptr;
  return L;
}

ff_status launch_sift_kd_query(const SiftLevel &L, const SiftKdQuery &Q, int r, int nw4,
                               cudaStream_t st) {
  const int G = L.Gx * L.Gy;
  FF_DISPATCH_SIFT(r, nw4, k_sift_kd_query, grid_blocks((long long)G * SIFT_GROUP), 256, 0, st, L,
                   Q);
  return FF_OK;
}

// Seeding (if L.flow_coarse), then 4 passes with n_rs random searches; the
// state starts and ends in (fa, ca), (fb, cb) is the other buffer.
ff_status run_sift_level(const SiftLevel &L, int r, int nw4, uint32_t *fa, int32_t *ca,
                         uint32_t *fb, int32_t *cb, int tile, int n_rs, int R, uint64_t seed,
                         cudaStream_t st) {
  const int G = L.Gx * L.Gy;
  const int blocks = grid_blocks((long long)G * SIFT_GROUP);
  if (L.flow_coarse) FF_DISPATCH_SIFT(r, nw4, k_sift_seed, blocks, 256, 0, st, L, fa, ca);
  int level = 0;
  while ((1 << level) < L.n) level++;
  SiftLevel Lp = L;  // the pass kernels count their evaluations when profiling
  Lp.evals = prof_evals(r, level);
  uint32_t *f[2] = {fa, fb};
  int32_t *c[2] = {ca, cb};
  for (int s = 0; s < 4; s++) {
    const int off = (s & 1) * (tile / 2);
    const int ntiles = ((L.Gx + off + tile - 1) / tile) * ((L.Gy + off + tile - 1) / tile);
    if (prof_enabled()) prof_begin(st, level);
    FF_DISPATCH_SIFT(r, nw4, k_sift_pass, ntiles, SIFT_GROUP * tile, 0, st, Lp, f[s & 1],
                     c[s & 1], f[(s + 1) & 1], c[(s + 1) & 1], s, tile);
    if (prof_enabled()) prof_end(st);
    if (s < 3 && s < n_rs)
      FF_DISPATCH_SIFT(r, nw4, k_sift_rs, blocks, 256, 0, st, L, f[(s + 1) & 1], c[(s + 1) & 1],
                       s, level, R * L.n, seed);
  }
  return FF_OK;
}

// ------------------------------------------------------------- whole path ----
constexpr int SIFT_MAXLV = 5;

struct SiftPlan {
  uint8_t *lab[2];
  uint8_t *desc[2];
  uint8_t *col[2][2];     // [colour set][frame] full-resolution colour groups
  uint8_t *col_n[2][2];   // the same smoothed at the current level
  uint8_t *down[2][2], *hbuf[2][2];  // smoothing scratch per (set, frame): one slice per group
  size_t down_stride, h_stride;      // bytes per group slice
  uint4 *K[SIFT_MAXLV][2][2];        // [level][colour set][frame] packed colours
  int32_t *feat[3], *qfeat[3];
  int32_t *perm[3], *split_dim[3], *split_val[3];
  KdBuild kd[3];
  uint32_t *fl[3][3];     // per flow: three flow buffers (coarse, current, other)
  int32_t *cs[3][3];
  void *filter_scratch;
  KdBuild *d_kd;
  PyrJob *d_jobs;         // per level: the smoothing jobs (one per colour group and frame)
};

static int sift_groups(const int Ss[2]) { return 2 * (Ss[0] / 3 + Ss[1] / 3); }

static void plan_sift(Arena &a, int W, int H, const ff_params *p, int S1, int S2, SiftPlan &P) {
  const size_t N = (size_t)W * H;
  const int Ss[2] = {S1, S2};
  a.take<char>(WS_HEADER);
  for (int f = 0; f < 2; f++) P.lab[f] = p->color == 1 ? a.take<uint8_t>(N * 3) : nullptr;
  for (int f = 0; f < 2; f++) P.desc[f] = a.take<uint8_t>(N * SIFT_DIM);
  // smoothing scratch of one group at the finest smoothed level (n = 2) bounds all
  const int Wc = (W + 1) / 2, Hc = (H + 1) / 2;
  P.down_stride = ((size_t)Wc * Hc * 3 + 255) & ~(size_t)255;
  P.h_stride = ((size_t)Hc * W * 3 * sizeof(int32_t) + 255) & ~(size_t)255;
  for (int c = 0; c < 2; c++)
    for (int f = 0; f < 2; f++) {
      P.col[c][f] = a.take<uint8_t>(N * Ss[c]);
      P.col_n[c][f] = a.take<uint8_t>(N * Ss[c]);
      if (p->k > 0) {
        P.down[c][f] = a.take<uint8_t>(P.down_stride * (Ss[c] / 3));
        P.hbuf[c][f] = a.take<uint8_t>(P.h_stride * (Ss[c] / 3));
      } else {
        P.down[c][f] = P.hbuf[c][f] = nullptr;
      }
    }
  for (int lv = 0; lv <= p->k; lv++)
    for (int c = 0; c < 2; c++)
      for (int f = 0; f < 2; f++) P.K[lv][c][f] = a.take<uint4>(N * sift_nw4(Ss[c]));
  const int ntop = 1 << p->k;
  const size_t Gtop = (size_t)((W + ntop - 1) / ntop) * ((H + ntop - 1) / ntop);
  const int D = kd_depth((int)N, p->leaf);
  for (int j = 0; j < 3; j++) {
    P.feat[j] = a.take<int32_t>(N * FEAT_PACKED_WORDS);
    P.qfeat[j] = a.take<int32_t>(Gtop * FEAT_STRIDE);
    P.perm[j] = a.take<int32_t>(N);
    P.split_dim[j] = a.take<int32_t>((size_t)1 << D);
    P.split_val[j] = a.take<int32_t>((size_t)1 << D);
    KdBuild &b = P.kd[j];
    b = KdBuild{};
    b.N = (int)N;
    b.leaf = p->leaf;
    {
      const int rj = j == 2 ? p->r2 : p->r;
      const long long span = (long long)(2 * rj + 1) * (2 * rj + 1) * 255;
      int vb = 0;
      while ((1ll << vb) <= span) vb++;
      b.value_bits = vb;
    }
    kd_bind_scratch(b, a);
    b.feat = P.feat[j];
    b.packed = 1;
    b.perm = P.perm[j];
    b.split_dim = P.split_dim[j];
    b.split_val = P.split_val[j];
    b.status = (DeviceStatus *)a.base;
    for (int i = 0; i < 3; i++) {
      P.fl[j][i] = a.take<uint32_t>(N);
      P.cs[j][i] = a.take<int32_t>(N);
    }
  }
  P.filter_scratch = a.take<char>(filter_scratch_bytes(W, H));
  P.d_kd = a.take<KdBuild>(3);
  P.d_jobs = a.take<PyrJob>((size_t)SIFT_MAXLV * sift_groups(Ss));
}

// The packed colours of every level: per level n > 1 every colour group of both
// frames smoothed like I^n in one batched launch sequence, then packed.
static ff_status sift_pyramid(const SiftPlan &P, int W, int H, int k, const int Ss[2],
                              cudaStream_t st) {
  const size_t N = (size_t)W * H;
  const int ng = sift_groups(Ss);
  for (int lv = 0; lv <= k; lv++) {
    const int n = 1 << lv;
    if (n > 1) {
      std::vector<PyrJob> jobs;
      for (int c = 0; c < 2; c++)
        for (int f = 0; f < 2; f++)
          for (int g = 0; g < Ss[c] / 3; g++) {
            PyrJob j{};
            j.img = P.col[c][f] + (size_t)g * N * 3;
            j.down = P.down[c][f] + P.down_stride * g;
            j.h = (int32_t *)(P.hbuf[c][f] + P.h_stride * g);
            j.sm = P.col_n[c][f] + (size_t)g * N * 3;
            j.W = W;
            j.H = H;
            jobs.push_back(j);
          }
      FF_TRY(launch_smooth_batch(jobs.data(), P.d_jobs + (size_t)lv * ng, (int)jobs.size(), n, st));
    }
    for (int c = 0; c < 2; c++)
      for (int f = 0; f < 2; f++)
        FF_TRY(launch_sift_pack(n > 1 ? P.col_n[c][f] : P.col[c][f], (int)N, Ss[c], P.K[lv][c][f],
                                st));
  }
  return FF_OK;
}

static ff_status run_sift_pair(const uint8_t *I1_in, const uint8_t *I2_in, int W, int H,
                               const ff_params *p, const int16_t *B[2], const int32_t *O[2],
                               const int Ss[2], int16_t *flows, uint8_t *valid, int32_t *err_sum,
                               int32_t *sparse, int32_t *n_sparse, uint8_t *mask, void *ws,
                               size_t ws_bytes, cudaStream_t st) {
  SiftPlan P;
  Arena a(ws, ws_bytes);
  plan_sift(a, W, H, p, Ss[0], Ss[1], P);
  if (!a.fits()) return FF_ERR_WORKSPACE;
  FF_TRY(clear_status(ws, st));
  const size_t N = (size_t)W * H;
  const uint8_t *I1 = I1_in, *I2 = I2_in;
  if (p->color == 1) {
    FF_TRY(launch_rgb_to_lab(I1_in, W, H, P.lab[0], st));
    FF_TRY(launch_rgb_to_lab(I2_in, W, H, P.lab[1], st));
    I1 = P.lab[0];
    I2 = P.lab[1];
  }
  const bool serial = exec_params().serial_flows != 0;
  const int k = p->k, ntop = 1 << k;
  // SIFT vectors of the input frames, their colours under both bases and the
  // colour pyramid on a side stream, beside the WHT features and the three kd
  // trees (one launch chain) on the caller's stream
  {
    SideSection pre;
    if (!serial) FF_TRY(pre.begin(st, 1));
    const cudaStream_t cs = serial ? st : pre.side[0];
    const uint8_t *in[2] = {I1_in, I2_in};
    for (int f = 0; f < 2; f++) {
      FF_TRY(launch_sift_descriptors(in[f], W, H, P.desc[f], cs));
      for (int c = 0; c < 2; c++)
        FF_TRY(launch_sift_colors(P.desc[f], (int)N, B[c], O[c], Ss[c], P.col[c][f], cs));
    }
    FF_TRY(sift_pyramid(P, W, H, k, Ss, cs));
    const int srcf[3] = {0, 1, 1}, tgtf[3] = {1, 0, 0}, rad[3] = {p->r, p->r, p->r2};
    const uint8_t *img[2] = {I1, I2};
    for (int j = 0; j < 3; j++) {
      FF_TRY(launch_features(img[tgtf[j]], W, H, rad[j], nullptr, 0, 1, P.feat[j], st, true));
      FF_TRY(launch_features(img[srcf[j]], W, H, rad[j], nullptr, 0, ntop, P.qfeat[j], st));
    }
    FF_TRY(launch_kd_build(P.kd, P.d_kd, 3, st));
    if (!serial) FF_TRY(pre.end());
  }
  // flows: forward I1 -> I2 (r, set 0), backward I2 -> I1 (r, set 0), (r2, set 1),
  // each flow's kd query and levels on a stream of its own
  const int srcf[3] = {0, 1, 1}, tgtf[3] = {1, 0, 0}, rad[3] = {p->r, p->r, p->r2};
  const int cset[3] = {0, 0, 1};
  SideSection sec;
  if (!serial) FF_TRY(sec.begin(st, 2));
  int cur[3] = {0, 0, 0};
  for (int j = 0; j < 3; j++) {
    const cudaStream_t fs = (serial || j == 0) ? st : sec.side[j - 1];
    const int c = cset[j], nw4 = sift_nw4(Ss[c]);
    for (int lv = k; lv >= 0; lv--) {
      const int n = 1 << lv;
      // three buffers per flow: the coarser level's final state, this level's
      // state and its ping-pong partner
      const int a0 = lv == k ? 0 : (cur[j] + 1) % 3, b0 = (a0 + 1) % 3;
      const uint32_t *coarse = lv == k ? nullptr : P.fl[j][cur[j]];
      SiftLevel L = make_sift_level(P.K[lv][c][srcf[j]], P.K[lv][c][tgtf[j]], W, H, n, j, coarse);
      if (lv == k) {
        SiftKdQuery Q;
        Q.perm = P.perm[j];
        Q.split_dim = P.split_dim[j];
        Q.split_val = P.split_val[j];
        Q.N = (int)N;
        Q.D = kd_depth((int)N, p->leaf);
        Q.qfeat = P.qfeat[j];
        Q.flow = P.fl[j][a0];
        Q.cost = P.cs[j][a0];
        Q.status = (DeviceStatus *)ws;
        FF_TRY(launch_sift_kd_query(L, Q, rad[j], nw4, fs));
      }
      FF_TRY(run_sift_level(L, rad[j], nw4, P.fl[j][a0], P.cs[j][a0], P.fl[j][b0], P.cs[j][b0],
                            p->tile, p->n_rs, p->R, p->seed, fs));
      cur[j] = a0;
    }
    if (cudaMemcpyAsync(flows + 2 * N * j, P.fl[j][cur[j]], N * sizeof(uint32_t),
                        cudaMemcpyDeviceToDevice, fs) != cudaSuccess)
      return FF_ERR_CUDA;
  }
  if (!serial) FF_TRY(sec.end());
  return launch_filter((const uint32_t *)flows, (const uint32_t *)(flows + 2 * N),
                       (const uint32_t *)(flows + 4 * N), W, H, p->eps, p->e, p->s, 1, valid,
                       err_sum, sparse, n_sparse, mask, P.filter_scratch, st);
}

// ------------------------------------------------------- per-level entries ---
struct SiftLevelWs {
  uint4 *Ks, *Kt;
  int32_t *qfeat;
  uint32_t *fb;
  int32_t *cb;
};
static SiftLevelWs bind_sift_level(Arena &a, int W, int H, int n, int S) {
  const size_t N = (size_t)W * H, G = (size_t)((W + n - 1) / n) * ((H + n - 1) / n);
  a.take<char>(WS_HEADER);
  SiftLevelWs L;
  L.Ks = a.take<uint4>(N * sift_nw4(S));
  L.Kt = a.take<uint4>(N * sift_nw4(S));
  L.qfeat = a.take<int32_t>(G * FEAT_STRIDE);
  L.fb = a.take<uint32_t>(G);
  L.cb = a.take<int32_t>(G);
  return L;
}

}  // namespace ff

using namespace ff;

extern "C" {

ff_status ff_sift_descriptors(const uint8_t *img, int W, int H, uint8_t *desc, void *stream) {
  FF_TRY(check_shape(W, H));
  if (!img || !desc || !aligned(desc, 16)) return FF_ERR_INVALID_ARG;
  return launch_sift_descriptors(img, W, H, desc, (cudaStream_t)stream);
}

ff_status ff_sift_moments(const uint8_t *desc, int N, uint64_t *sum, uint64_t *gram,
                          void *stream) {
  if (N < 0 || (N > 0 && (!desc || !sum || !gram)) || !aligned(desc, 16) || !aligned(sum, 8) ||
      !aligned(gram, 8))
    return FF_ERR_INVALID_ARG;
  return launch_sift_moments(desc, N, (unsigned long long *)sum, (unsigned long long *)gram,
                             (cudaStream_t)stream);
}

ff_status ff_sift_pca_workspace_size(size_t *bytes) {
  if (!bytes) return FF_ERR_INVALID_ARG;
  Arena a;
  a.take<char>(WS_HEADER);
  a.take<double>((size_t)SIFT_DIM * SIFT_DIM);
  *bytes = a.off;
  return FF_OK;
}

ff_status ff_sift_pca(const uint64_t *sum, const uint64_t *gram, int64_t count, int S,
                      int16_t *basis, int32_t *offset, double *eigval, void *ws, size_t ws_bytes,
                      void *stream) {
  if (!sum || !gram || !basis || !offset || count <= 0 || !sift_S_ok(S)) return FF_ERR_INVALID_ARG;
  if (!aligned(sum, 8) || !aligned(gram, 8) || !aligned(basis, 2) || !aligned(offset, 4) ||
      (eigval && !aligned(eigval, 8)))
    return FF_ERR_INVALID_ARG;
  size_t need;
  FF_TRY(ff_sift_pca_workspace_size(&need));
  FF_TRY(check_ws(ws, ws_bytes, need));
  cudaStream_t st = (cudaStream_t)stream;
  FF_TRY(clear_status(ws, st));
  Arena a(ws, ws_bytes);
  a.take<char>(WS_HEADER);
  double *VT = a.take<double>((size_t)SIFT_DIM * SIFT_DIM);
  return launch_sift_pca((const unsigned long long *)sum, (const unsigned long long *)gram, count,
                         S, VT, basis, offset, eigval, (DeviceStatus *)ws, st);
}

ff_status ff_sift_colors(const uint8_t *desc, int W, int H, const int16_t *basis,
                         const int32_t *offset, int S, uint8_t *colors, void *stream) {
  FF_TRY(check_shape(W, H));
  if (!desc || !basis || !offset || !colors || !sift_S_ok(S) || !aligned(desc, 16))
    return FF_ERR_INVALID_ARG;
  return launch_sift_colors(desc, W * H, basis, offset, S, colors, (cudaStream_t)stream);
}

ff_status ff_sift_level_workspace_size(int W, int H, int n, int S, size_t *bytes) {
  FF_TRY(check_shape(W, H));
  if (!bytes || !pow2_upto(n, 16) || !sift_S_ok(S)) return FF_ERR_INVALID_ARG;
  Arena a;
  bind_sift_level(a, W, H, n, S);
  *bytes = a.off;
  return FF_OK;
}

ff_status ff_sift_kdtree_init(const int32_t *perm, const int32_t *split_dim,
                              const int32_t *split_val, int leaf, const uint8_t *src_img,
                              const uint8_t *colors_src, const uint8_t *colors_tgt, int S, int W,
                              int H, int n, int r, int16_t *flow, int32_t *cost, void *ws,
                              size_t ws_bytes, void *stream) {
  FF_TRY(check_shape(W, H));
  if (!perm || !split_dim || !split_val || !src_img || !colors_src || !colors_tgt || !flow ||
      !cost || !aligned(flow, 4) || !aligned(cost, 4))
    return FF_ERR_INVALID_ARG;
  if (leaf < 2 || leaf > 32 || !pow2_upto(n, 16) || r < 1 || r > PLANE_PAD || !sift_S_ok(S))
    return FF_ERR_INVALID_ARG;
  size_t need;
  FF_TRY(ff_sift_level_workspace_size(W, H, n, S, &need));
  FF_TRY(check_ws(ws, ws_bytes, need));
  cudaStream_t st = (cudaStream_t)stream;
  Arena a(ws, ws_bytes);
  SiftLevelWs Lw = bind_sift_level(a, W, H, n, S);
  FF_TRY(clear_status(ws, st));
  const int N = W * H;
  FF_TRY(launch_sift_pack(colors_src, N, S, Lw.Ks, st));
  FF_TRY(launch_sift_pack(colors_tgt, N, S, Lw.Kt, st));
  FF_TRY(launch_features(src_img, W, H, r, nullptr, 0, n, Lw.qfeat, st));
  SiftLevel L = make_sift_level(Lw.Ks, Lw.Kt, W, H, n, 0, nullptr);
  SiftKdQuery Q;
  Q.perm = perm;
  Q.split_dim = split_dim;
  Q.split_val = split_val;
  Q.N = N;
  Q.D = kd_depth(N, leaf);
  Q.qfeat = Lw.qfeat;
  Q.flow = (uint32_t *)flow;
  Q.cost = cost;
  Q.status = (DeviceStatus *)ws;
  return launch_sift_kd_query(L, Q, r, sift_nw4(S), st);
}

ff_status ff_sift_search_level(const uint8_t *colors_src, const uint8_t *colors_tgt, int S, int W,
                               int H, int n, int r, const int16_t *flow_coarse, const ff_params *p,
                               int flow_id, int16_t *flow, int32_t *cost, void *ws,
                               size_t ws_bytes, void *stream) {
  FF_TRY(check_shape(W, H));
  FF_TRY(check_params(p));
  if (p->subpel != 1) return FF_ERR_INVALID_ARG;
  if (!colors_src || !colors_tgt || !flow || !cost || !aligned(flow, 4) || !aligned(cost, 4))
    return FF_ERR_INVALID_ARG;
  if (flow_coarse && !aligned(flow_coarse, 4)) return FF_ERR_INVALID_ARG;
  if (!pow2_upto(n, 16) || r < 1 || r > PLANE_PAD || flow_id < 0 || flow_id > 3 || !sift_S_ok(S))
    return FF_ERR_INVALID_ARG;
  size_t need;
  FF_TRY(ff_sift_level_workspace_size(W, H, n, S, &need));
  FF_TRY(check_ws(ws, ws_bytes, need));
  cudaStream_t st = (cudaStream_t)stream;
  Arena a(ws, ws_bytes);
  SiftLevelWs Lw = bind_sift_level(a, W, H, n, S);
  FF_TRY(clear_status(ws, st));
  const int N = W * H;
  FF_TRY(launch_sift_pack(colors_src, N, S, Lw.Ks, st));
  FF_TRY(launch_sift_pack(colors_tgt, N, S, Lw.Kt, st));
  SiftLevel L = make_sift_level(Lw.Ks, Lw.Kt, W, H, n, flow_id, (const uint32_t *)flow_coarse);
  return run_sift_level(L, r, sift_nw4(S), (uint32_t *)flow, cost, Lw.fb, Lw.cb, p->tile, p->n_rs,
                        p->R, p->seed, st);
}

ff_status ff_sift_workspace_size(int W, int H, const ff_params *p, int S1, int S2, size_t *bytes) {
  FF_TRY(check_shape(W, H));
  FF_TRY(check_params(p));
  if (!bytes || !sift_S_ok(S1) || !sift_S_ok(S2)) return FF_ERR_INVALID_ARG;
  SiftPlan P;
  Arena a;
  plan_sift(a, W, H, p, S1, S2, P);
  *bytes = a.off;
  return FF_OK;
}

ff_status ff_sift_flow_fields(const uint8_t *I1, const uint8_t *I2, int W, int H,
                              const ff_params *p, const int16_t *basis1, const int32_t *offset1,
                              int S1, const int16_t *basis2, const int32_t *offset2, int S2,
                              int16_t *flows, uint8_t *valid, int32_t *err_sum, int32_t *sparse,
                              int32_t *n_sparse, uint8_t *mask, void *ws, size_t ws_bytes,
                              void *stream) {
  FF_TRY(check_shape(W, H));
  FF_TRY(check_params(p));
  if (p->subpel != 1) return FF_ERR_INVALID_ARG;
  if (!I1 || !I2 || !basis1 || !offset1 || !basis2 || !offset2 || !flows || !valid || !err_sum ||
      !sparse || !n_sparse || !mask || !aligned(flows, 4))
    return FF_ERR_INVALID_ARG;
  if (!sift_S_ok(S1) || !sift_S_ok(S2)) return FF_ERR_INVALID_ARG;
  size_t need;
  FF_TRY(ff_sift_workspace_size(W, H, p, S1, S2, &need));
  FF_TRY(check_ws(ws, ws_bytes, need));
  const int16_t *B[2] = {basis1, basis2};
  const int32_t *O[2] = {offset1, offset2};
  const int Ss[2] = {S1, S2};
  return run_sift_pair(I1, I2, W, H, p, B, O, Ss, flows, valid, err_sum, sparse, n_sparse, mask,
                       ws, ws_bytes, (cudaStream_t)stream);
}

}  // extern "C"
