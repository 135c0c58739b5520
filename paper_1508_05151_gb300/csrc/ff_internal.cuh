// Internal declarations of the GB300 Flow Fields library. Not part of the ABI.
//
// Data layout in HBM
//   Census "phase planes". At spacing n the census image of a frame is stored as
//   n*n planes, one per pixel phase (x mod n, y mod n). Plane (px, py) entry
//   (i, j) holds the census of pixel (clamp(px + n*(i - P)), clamp(py + n*(j - P)))
//   for i in [0, NX + 2P), j in [0, NY + 2P), NX = ceil(W/n), NY = ceil(H/n),
//   P >= the largest patch radius. The taps of a subsampled patch P^n_r around
//   any pixel (Eq. 3) then form a dense (2r+1)^2 block of one plane, already
//   clamped at the image border, so every tap is a plain in-bounds load and each
//   patch row is 2r+1 consecutive words. The row pitch is a multiple of 16 bytes.
//
//   Flows are packed int16 pairs in one uint32 (dx in the low half); costs int32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "flowfields.h"

namespace ff {

constexpr int32_t COST_UNSET = 0x7fffffff;
constexpr int NFEAT = 27;
constexpr int FEAT_STRIDE = 28;  // int32 per feature row (27 + pad) = 112 bytes

// Packed feature rows (the kd build's target features on the flow path): value j
// of a row, biased by 2^17 to an unsigned 18-bit field, at bits [18 j, 18 j + 18)
// of 16 32-bit words (64 bytes). Exact for |value| < 2^17; WHT features of radius
// r <= 8 stay within (2r+1)^2 * 255 = 73,695.
constexpr int FEAT_PACKED_WORDS = 16;
constexpr int FEAT_PACK_BITS = 18, FEAT_PACK_BIAS = 1 << 17;
constexpr uint32_t FEAT_PACK_MASK = (1u << FEAT_PACK_BITS) - 1u;

__host__ __device__ __forceinline__ void pack_feat_row(const int32_t *v, uint32_t *w) {
#pragma unroll
  for (int i = 0; i < FEAT_PACKED_WORDS; i++) w[i] = 0;
#pragma unroll
  for (int j = 0; j < NFEAT; j++) {
    const uint32_t u = (uint32_t)(v[j] + FEAT_PACK_BIAS) & FEAT_PACK_MASK;
    const int bit = FEAT_PACK_BITS * j, k = bit >> 5, o = bit & 31;
    w[k] |= u << o;
    if (o + FEAT_PACK_BITS > 32) w[k + 1] |= u >> (32 - o);
  }
}

__device__ __forceinline__ int32_t unpack_feat_field(uint32_t lo, uint32_t hi, int o) {
  return (int32_t)(__funnelshift_r(lo, hi, o) & FEAT_PACK_MASK) - FEAT_PACK_BIAS;
}

__device__ __forceinline__ void unpack_feat_row(const uint32_t *w, int32_t *v) {
#pragma unroll
  for (int j = 0; j < NFEAT; j++) {
    const int bit = FEAT_PACK_BITS * j, k = bit >> 5, o = bit & 31;
    v[j] = unpack_feat_field(w[k], o + FEAT_PACK_BITS > 32 ? w[k + 1] : 0u, o);
  }
}

// One value of a packed row (dim a run-time index).
__device__ __forceinline__ int32_t packed_feat_value(const uint32_t *row, int dim) {
  const int bit = FEAT_PACK_BITS * dim, k = bit >> 5, o = bit & 31;
  return unpack_feat_field(row[k], o + FEAT_PACK_BITS > 32 ? row[k + 1] : 0u, o);
}
constexpr int PLANE_PAD = 8;     // P: supports patch radii up to 8
constexpr int MAX_TILE = 32;
constexpr int MAX_K = 8;

// Device status word at the start of every workspace (16 bytes, first 256
// reserved): code, x, y, spare.
struct DeviceStatus {
  uint32_t code;
  int32_t x, y, spare;
};
constexpr size_t WS_HEADER = 256;
enum : uint32_t { DEV_OK = 0, DEV_ERR_BOUNDS = 1, DEV_ERR_KD = 2, DEV_ERR_TIMEOUT = 3 };

__device__ __forceinline__ void raise_status(DeviceStatus *st, uint32_t code, int x, int y) {
  if (st && atomicCAS(&st->code, 0u, code) == 0u) {
    st->x = x;
    st->y = y;
  }
}

// ---------------------------------------------------------------- flows ------
__host__ __device__ __forceinline__ uint32_t pack_flow(int dx, int dy) {
  return (uint32_t)(uint16_t)(int16_t)dx | ((uint32_t)(uint16_t)(int16_t)dy << 16);
}
__host__ __device__ __forceinline__ int flow_dx(uint32_t f) { return (int)(int16_t)(f & 0xffffu); }
__host__ __device__ __forceinline__ int flow_dy(uint32_t f) { return (int)(int16_t)(f >> 16); }

__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// ---------------------------------------------------------------- planes -----
// With subpixel flows (q = params.subpel > 1, flows in units of 1/q pixel) a
// frame carries the census of its image interpolated at each subpixel phase
// (a, b) = (X mod q, Y mod q) of a target X = q x + a, Y = q y + b: the planes of
// phase (a, b) follow those of the phases before it, plane index
// (b q + a) n^2 + (py n + px). Phase (0, 0) is the plain census, so integer
// positions (every source patch, every q = 1 target) use the first n^2 planes.
struct Planes {
  uint32_t *base;  // plane (px, py) at base + (py * n + px) * plane_words
  int W, H, n, log2n;
  int q, log2q;     // subpixel phases per axis (1, 2, 4)
  int NX, NY;       // ceil(W/n), ceil(H/n)
  int pitch;        // words per padded row (>= NX + 2P, multiple of 4)
  int rows;         // NY + 2P
  size_t plane_words;  // pitch * rows
  // Transposed copy of every plane (row = x entry, column = y entry), so that a
  // vertical run of taps is contiguous too.
  uint32_t *baseT;
  int pitchT;          // >= NY + 2P, multiple of 4
  size_t plane_wordsT;  // pitchT * (NX + 2P)
};

__host__ __device__ inline Planes make_planes(uint32_t *base, int W, int H, int n, int q = 1) {
  Planes p;
  p.base = base;
  p.W = W;
  p.H = H;
  p.n = n;
  int l = 0;
  while ((1 << l) < n) l++;
  p.log2n = l;
  p.q = q;
  p.log2q = q >= 4 ? 2 : (q >= 2 ? 1 : 0);
  p.NX = (W + n - 1) / n;
  p.NY = (H + n - 1) / n;
  p.pitch = ((p.NX + 2 * PLANE_PAD) + 3) & ~3;
  p.rows = p.NY + 2 * PLANE_PAD;
  p.plane_words = (size_t)p.pitch * p.rows;
  p.pitchT = ((p.NY + 2 * PLANE_PAD) + 3) & ~3;
  p.plane_wordsT = (size_t)p.pitchT * (p.NX + 2 * PLANE_PAD);
  p.baseT = base ? base + p.plane_words * (size_t)n * n * q * q : nullptr;
  return p;
}
__host__ __device__ inline size_t planes_words(int W, int H, int n, int q = 1) {
  Planes p = make_planes(nullptr, W, H, n);
  return (p.plane_words + p.plane_wordsT) * (size_t)n * n * q * q;
}
// The n^2 planes of subpixel phase ph (= b q + a) as a plane set of their own
// (for writing them).
__host__ __device__ inline Planes phase_view(const Planes &P, int ph) {
  Planes v = P;
  const size_t per = (size_t)P.n * P.n;
  v.base = P.base + per * P.plane_words * ph;
  v.baseT = P.baseT + per * P.plane_wordsT * ph;
  v.q = 1;
  v.log2q = 0;
  return v;
}

// Address of the centre tap of the patch around pixel (x, y), inside the image.
__device__ __forceinline__ const uint32_t *plane_centre(const Planes &P, int x, int y) {
  int m = P.n - 1;
  const uint32_t *pl = P.base + (size_t)(((y & m) << P.log2n) + (x & m)) * P.plane_words;
  return pl + (size_t)((y >> P.log2n) + PLANE_PAD) * P.pitch + (x >> P.log2n) + PLANE_PAD;
}

// Plane index and entry of the target (X, Y) in units of 1/q pixel (X, Y >= 0
// inside the image; for q = 1 the pixel itself).
// lq = P.log2q, passed explicitly so that a caller that knows q = 1 at compile
// time (lq a constant 0) drops the phase arithmetic.
__device__ __forceinline__ void target_plane_lq(const Planes &P, int X, int Y, int lq, int &ph,
                                                int &ex, int &ey) {
  const int m = P.n - 1, qm = (1 << lq) - 1;
  const int x = X >> lq, y = Y >> lq;
  ph = ((((Y & qm) << lq) + (X & qm)) << (2 * P.log2n)) + ((y & m) << P.log2n) + (x & m);
  ex = (x >> P.log2n) + PLANE_PAD;
  ey = (y >> P.log2n) + PLANE_PAD;
}
__device__ __forceinline__ void target_plane(const Planes &P, int X, int Y, int &ph, int &ex,
                                             int &ey) {
  target_plane_lq(P, X, Y, P.log2q, ph, ex, ey);
}
__device__ __forceinline__ const uint32_t *target_centre(const Planes &P, int X, int Y) {
  int ph, ex, ey;
  target_plane(P, X, Y, ph, ex, ey);
  return P.base + (size_t)ph * P.plane_words + (size_t)ey * P.pitch + ex;
}
// Candidate flow (dx, dy) (units of 1/q pixel) at pixel (px, py) with its target
// clamped into the image: X = clamp(q px + dx, 0, q (W - 1)), likewise Y; returns
// the clamped flow, packed.
__device__ __forceinline__ uint32_t clamp_target_lq(const Planes &P, int px, int py, int dx,
                                                    int dy, int lq, int &X, int &Y) {
  X = clampi((px << lq) + dx, 0, (P.W - 1) << lq);
  Y = clampi((py << lq) + dy, 0, (P.H - 1) << lq);
  return pack_flow(X - (px << lq), Y - (py << lq));
}
__device__ __forceinline__ uint32_t clamp_target(const Planes &P, int px, int py, int dx, int dy,
                                                 int &X, int &Y) {
  return clamp_target_lq(P, px, py, dx, dy, P.log2q, X, Y);
}
__device__ __forceinline__ uint32_t clamp_target(const Planes &P, int px, int py, uint32_t f,
                                                 int &X, int &Y) {
  return clamp_target(P, px, py, flow_dx(f), flow_dy(f), X, Y);
}

// ------------------------------------------------------- patch cost ---------
// E_d over the (2R+1)^2 taps of P^n_r (Eq. 3) with the census data term: a group
// of 16 lanes (one half warp, mask gmask) splits the taps, tap t = lane + 16k in
// row-major patch order, and the popcounts are summed with xor shuffles. Both
// operands are given as the address of the patch centre and a row pitch in
// words; the result is complete in every lane of the group.
template <int R>
__device__ __forceinline__ int group_cost(const uint32_t *sc, int spitch, const uint32_t *tc,
                                          int tpitch, int l16, unsigned gmask) {
  constexpr int L = 2 * R + 1, LL = L * L, KT = (LL + 15) / 16;
  int acc = 0;
#pragma unroll
  for (int k = 0; k < KT; k++) {
    const int t = l16 + 16 * k;
    if (t < LL) {
      const int v = t / L - R, u = t % L - R;
      acc += __popc(sc[v * spitch + u] ^ __ldg(tc + v * tpitch + u));
    }
  }
  acc += __shfl_xor_sync(gmask, acc, 8);
  acc += __shfl_xor_sync(gmask, acc, 4);
  acc += __shfl_xor_sync(gmask, acc, 2);
  acc += __shfl_xor_sync(gmask, acc, 1);
  return acc;
}

#define FF_DISPATCH_R(r, ...)                   \
  switch (r) {                                  \
    case 1: { constexpr int RR = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int RR = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int RR = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int RR = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int RR = 5; __VA_ARGS__; } break; \
    case 6: { constexpr int RR = 6; __VA_ARGS__; } break; \
    case 7: { constexpr int RR = 7; __VA_ARGS__; } break; \
    case 8: { constexpr int RR = 8; __VA_ARGS__; } break; \
    default: return FF_ERR_INVALID_ARG;         \
  }

// ------------------------------------------------------ descriptors ----------
// Kernels read their problem descriptors from device memory. They are written
// there, on the stream, by a small kernel that receives them as parameters.
template <typename T, int CAP>
struct DescChunk {
  T d[CAP];
};
template <typename T, int CAP>
__global__ void k_write_desc(DescChunk<T, CAP> c, int n, T *dst) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = c.d[i];
}
void count_launch(int n);
template <typename T>
inline ff_status upload_desc(const T *host, T *dev, int n, cudaStream_t st) {
  constexpr int CAP = (3072 / sizeof(T)) > 0 ? (3072 / sizeof(T)) : 1;
  for (int i = 0; i < n; i += CAP) {
    DescChunk<T, CAP> c;
    int m = n - i < CAP ? n - i : CAP;
    for (int k = 0; k < m; k++) c.d[k] = host[i + k];
    k_write_desc<T, CAP><<<1, 32, 0, st>>>(c, m, dev + i);
    count_launch(1);
    if (cudaPeekAtLastError() != cudaSuccess) {
      (void)cudaGetLastError();
      return FF_ERR_CUDA;
    }
  }
  return FF_OK;
}

// ------------------------------------------------------------- RNG ------------
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): golden-gamma increment, then the
// 64-bit finaliser. Key layout: gx bits 0-23, gy 24-47, step 48-49, log2 n 50-52,
// flow id 53-54, xored into the seed. Lemire's multiply-shift maps the low and
// high 32-bit halves to [0, 2 Rn] for dx and dy.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ void rs_offset(uint64_t seed, int flow_id, int level, int step,
                                                   int gx, int gy, int Rn, int &dx, int &dy) {
  uint64_t key = seed ^ ((uint64_t)gx & 0xffffffULL) ^ (((uint64_t)gy & 0xffffffULL) << 24) ^
                 ((uint64_t)(step & 3) << 48) ^ ((uint64_t)(level & 7) << 50) ^
                 ((uint64_t)(flow_id & 3) << 53);
  uint64_t z = splitmix64(key);
  uint64_t span = 2ull * (uint64_t)Rn + 1ull;
  dx = (int)(((z & 0xffffffffULL) * span) >> 32) - Rn;
  dy = (int)(((z >> 32) * span) >> 32) - Rn;
}

// --------------------------------------------------------- workspace ---------
// Bump allocator over the caller's workspace; with base == nullptr it only
// measures. Every block is 256-byte aligned.
struct Arena {
  char *base;
  size_t cap, off;
  explicit Arena(void *b = nullptr, size_t c = 0) : base((char *)b), cap(c), off(0) {}
  template <typename T>
  T *take(size_t count) {
    size_t bytes = ((count * sizeof(T)) + 255) & ~(size_t)255;
    T *p = base ? (T *)(base + off) : nullptr;
    off += bytes;
    return p;
  }
  bool fits() const { return base == nullptr || off <= cap; }
};

// ------------------------------------------------------- host-side checks ---
// Parameter and image-shape checks shared by every entry point.
ff_status check_params(const ff_params *p);
ff_status check_shape(int W, int H);
inline bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }
inline bool pow2_upto(int n, int hi) { return n >= 1 && n <= hi && (n & (n - 1)) == 0; }
// The caller's workspace: present, 256-byte aligned and at least `need` bytes.
inline ff_status check_ws(void *ws, size_t have, size_t need) {
  if (need == 0) return FF_OK;
  if (!ws || !aligned(ws, 256)) return FF_ERR_WORKSPACE;
  if (have < need) return FF_ERR_WORKSPACE;
  return FF_OK;
}
// Zeroes the device status word at the start of the workspace.
inline ff_status clear_status(void *ws, cudaStream_t st) {
  if (cudaMemsetAsync(ws, 0, sizeof(DeviceStatus), st) != cudaSuccess) return FF_ERR_CUDA;
  return FF_OK;
}

// Raises `func`'s dynamic shared-memory limit to at least `bytes` on the current
// device. The setting is per device and per kernel; it is remembered per
// (device, kernel) under a lock, so concurrent first calls from several host
// threads, or calls on several devices, each see the opt-in done before their
// launch. Returns FF_ERR_CUDA when the runtime refuses it.
ff_status smem_opt_in(const void *func, size_t bytes);

// ---------------------------------------------------- execution parameters ---
// Launch shapes that do not change results (set by the autotuner).
const ff_exec_params &exec_params();

// ------------------------------------------------------- launch accounting ---
constexpr int PROF_LEVELS = 5;  // levels n = 1, 2, 4, 8, 16 in the per-level profile
void count_launch(int n);
bool prof_enabled();
void prof_begin(cudaStream_t s, int tag);  // tag: log2 n of the launch's level
void prof_end(cudaStream_t s);
// Counter block [4] of the pass kernels' evaluations at radius r and level log2n
// when evaluation counting is on, else nullptr.
unsigned long long *prof_evals(int r, int log2n);

#define FF_CHECK_LAUNCH()                                     \
  do {                                                        \
    ::ff::count_launch(1);                                     \
    if (cudaPeekAtLastError() != cudaSuccess) {               \
      (void)cudaGetLastError();                               \
      return FF_ERR_CUDA;                                     \
    }                                                         \
  } while (0)

#define FF_TRY(expr)                      \
  do {                                    \
    ff_status _s = (expr);                \
    if (_s != FF_OK) return _s;           \
  } while (0)

// ------------------------------------------------------------ pyramid --------
struct LanczosTable {
  int32_t base[16];
  int32_t w[16][6];
};
void lanczos_table(int n, LanczosTable *t);  // host
size_t smooth_scratch_bytes(int W, int H, int n);
ff_status launch_smooth(const uint8_t *img, int W, int H, int n, uint8_t *out, void *scratch,
                        cudaStream_t st);
ff_status launch_census(const uint8_t *imgn, int W, int H, int n, uint32_t *out, cudaStream_t st);
// Census (spacing n) of imgn interpolated at subpixel phase (a, b) of q: the
// colours q^2-scaled bilinear sums of the pixel and its right, lower and
// lower-right neighbours (clamped), exact in integers.
ff_status launch_census_subpel(const uint8_t *imgn, int W, int H, int n, int q, int a, int b,
                               uint32_t *out, cudaStream_t st);
ff_status launch_planes(const uint32_t *census, Planes P, cudaStream_t st);
// One frame of one pair at one pyramid level (the batched pyramid): the frame,
// its scratch (area-down image, horizontal Lanczos pass, I^n, census) and the
// phase-0 view of its census planes at spacing n.
struct PyrJob {
  const uint8_t *img;
  uint8_t *down;
  int32_t *h;
  uint8_t *sm;
  uint32_t *census;
  Planes pl;
  int W, H;
};
// I^n (n > 1), its census and the phase planes of every job, one launch per step
// over all jobs. host/dev: the jobs (dev: device copy written on the stream).
ff_status launch_pyramid_level(const PyrJob *host, PyrJob *dev, int njobs, int n, cudaStream_t st);
// Only the smoothing steps of the jobs (img -> down -> h -> sm), n > 1.
ff_status launch_smooth_batch(const PyrJob *host, PyrJob *dev, int njobs, int n, cudaStream_t st);

// -------------------------------------------------------------- colour -------
ff_status launch_rgb_to_lab(const uint8_t *img, int W, int H, uint8_t *out, cudaStream_t st);

// ----------------------------------------------------------- features --------
// pts != NULL: explicit (x, y) list; else grid of spacing grid_n (1 = all pixels).
// packed (all pixels only): 16-word packed rows instead of [28] int32 rows.
ff_status launch_features(const uint8_t *img, int W, int H, int r, const int32_t *pts, int npts,
                          int grid_n, int32_t *feat, cudaStream_t st, bool packed = false);

// ------------------------------------------------------------- kd tree -------
struct KdBuild {
  const int32_t *feat;  // [N][28] int32, or [N][16] packed words when `packed`
  int packed;
  int N, leaf, D;
  int32_t *perm;        // [N] output
  int32_t *split_dim, *split_val;  // [2^D - 1]
  // scratch (from kd_scratch)
  int32_t *perm_tmp;
  int32_t *seg_off;    // offsets of all top-level segments
  int32_t *mm;         // min/max per top-level segment and dim (two levels)
  uint32_t *hist;      // radix histograms of the first digit
  int32_t *sel;        // per-segment select state (two levels)
  int32_t *cnt;        // per-segment partition counters (two levels)
  int32_t *ccnt;       // per-segment collected-key counts (two levels)
  int32_t *arrive;     // per-segment count of chunk CTAs done with the current step
  unsigned long long *keys;  // [N] select keys of the current level, by position
  unsigned long long *coll;  // [N] keys of each segment's median bucket, at the segment's positions
  int value_bits;      // bound on the bits of any dimension's spread (0: unknown)
  int top_levels;      // levels built by the multi-block path
  DeviceStatus *status;  // set if a partition count is inconsistent
};
int kd_depth(int N, int leaf);
size_t kd_scratch_bytes(int N, int leaf);
void kd_bind_scratch(KdBuild &b, Arena &a);
// Builds `ntrees` trees in the same launches.
ff_status launch_kd_build(const KdBuild *trees, KdBuild *dev_desc, int ntrees, cudaStream_t st);

struct KdQuery {
  const int32_t *perm, *split_dim, *split_val;
  int N, D, leaf;
  const int32_t *qfeat;     // [G][28] features of the grid points
  Planes src, tgt;          // level-n census planes
  int r;
  const uint32_t *proposals;  // [G][K] packed or nullptr
  int K;
  uint32_t *flow;  // [G]
  int32_t *cost;   // [G]
  DeviceStatus *status;  // DEV_ERR_BOUNDS: a split dimension or leaf entry out of range
};
ff_status launch_kd_query(const KdQuery *q, KdQuery *dev_desc, int nq, cudaStream_t st);

// Start of segment i of depth d when [0, N) is halved d times, the left half
// taking floor(m/2) (the kd tree's leaf ranges).
__host__ __device__ __forceinline__ int seg_begin(int N, int d, int i) {
  if (i >= (1 << d)) return N;
  int b = 0, e = N;
  for (int k = d - 1; k >= 0; k--) {
    int half = (e - b) >> 1;
    if ((i >> k) & 1) b += half;
    else e = b + half;
  }
  return b;
}

// -------------------------------------------------------------- search -------
struct SearchProblem {
  Planes src, tgt;   // level-n census planes of the source and target frame
  int r, flow_id;
  const uint32_t *flow_coarse;  // seeding input (level 2n grid) or nullptr
  uint32_t *flow_a, *flow_b;    // ping-pong state [G]
  int32_t *cost_a, *cost_b;
  uint32_t *flow_final;  // where the last pass writes (nullptr = ping-pong buffer)
  int32_t *cost_final;
};
// Seeds (if flow_coarse) and runs the 4 passes with n_rs random searches.
// After the call the state is in flow_final/cost_final when given, else in
// flow_a/cost_a.
// Problems of one patch radius, all on stream st (no side stream).
ff_status run_level_on(const SearchProblem *probs, SearchProblem *dev_desc, int nprob, int tile,
                       int n_rs, int R, uint64_t seed, cudaStream_t st);
// A fork/join section on the per-device side streams: begin() makes nside (1..3)
// side streams wait for the work enqueued so far on st, end() makes st wait
// for them. Two signal events order work between the streams inside the
// section: signal(k, s) marks the point reached on stream s, wait(k, s) makes s
// wait for it. Host threads are serialised between begin() and end(); the
// destructor ends an open section (error paths).
struct SideSection {
  cudaStream_t main = nullptr, side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t join[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t sig[2] = {nullptr, nullptr};
  bool locked = false;
  ff_status begin(cudaStream_t st, int nside);
  ff_status signal(int k, cudaStream_t s);
  ff_status wait(int k, cudaStream_t s);
  ff_status end();
  ~SideSection() {
    if (locked) end();
  }
};
// One persistent cooperative launch for the whole level of every problem (tile
// <= 16): seeding, four passes with the random searches, bounded grid barriers.
// tile_base: device int32 [2 (nprob + 1)] scratch; bar: a device counter.
ff_status run_level_persistent(const SearchProblem *probs, SearchProblem *dev_desc, int nprob,
                               int32_t *tile_base, unsigned *bar, DeviceStatus *status, int tile,
                               int n_rs, int R, uint64_t seed, cudaStream_t st);
// Test hooks of the bounded waits: the persistent kernel's barrier wait limit in
// clock cycles (0: the default) and a block that never reaches the first barrier
// (-1: none); net_stall > 0 makes every tcgen05 kernel of the net first wait that
// many polls on an mbarrier nothing completes (0: off).
void set_wait_test(long long budget_cycles, int skip_block, int net_stall);
int net_stall_polls();
ff_status run_level(const SearchProblem *probs, SearchProblem *dev_desc, int nprob, int tile,
                    int n_rs, int R, uint64_t seed, cudaStream_t st);

// -------------------------------------------------------------- filter -------
size_t filter_scratch_bytes(int W, int H);
// Flows in units of 1/q pixel (q = 1: pixels).
ff_status launch_filter(const uint32_t *F, const uint32_t *Fb1, const uint32_t *Fb2, int W, int H,
                        int eps, int e, int s, int q, uint8_t *valid, int32_t *err_sum,
                        int32_t *sparse, int32_t *n_sparse, uint8_t *mask, void *scratch,
                        cudaStream_t st);

}  // namespace ff
