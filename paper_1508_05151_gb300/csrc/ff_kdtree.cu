// Sec. 3.1: device kd tree over the 27-D WHT vectors of all target pixels, and
// the bounded-leaf query + rerank that gives the initial flow (Eq. 1 / Eq. 4).
//
// Tree definition (shared with the CPU statement of the method): perfect tree of
// depth D = min{d : ceil(N / 2^d) <= l}; a node of m points splits on the
// dimension of largest (max - min) (lowest index on ties); the first floor(m/2)
// points under the order (value, pixel index) go left; split value = value of the
// first right point. Segments of a level are contiguous in `perm`, obtained by
// halving [0, N) (left takes floor(m/2)).
//
// Feature rows come as int32 [28] (the public build) or packed 64-byte rows of
// 18-bit fields (the flow path; see ff_internal.cuh).
//
// Build, level by level:
//   top levels (segments > SUB_MAX points): three multi-CTA kernels per level,
//   each over chunks of KD_CHUNK positions. The CTA that finishes the last chunk
//   of a segment (a per-segment arrival count after a memory fence; nothing
//   waits) runs that segment's next step, so a level needs no further launches:
//     hist      key = (value - min) << ibits | pixel index (unique), cached per
//               position; 12-bit histogram of the key's top digit. Last CTA of a
//               segment: the bin holding the rank-floor(m/2) key.
//     collect   the keys in that bin are appended to the segment's list (stored
//               at the segment's own positions, so it always fits). Last CTA: the
//               exact key of the remaining rank in the list (bitonic sort in
//               shared memory; radix passes over the list when it is long, e.g.
//               for heavily tied features).
//     partition key < selected key -> left child, else right; the children's
//               per-dimension min/max. Last CTA: the children's split dimension
//               and key width (the next level's select state).
//   The per-level state (select state, counters, min/max) alternates between two
//   buffers by level parity, so a segment that finished can prepare its children
//   while other segments of the level are still being partitioned. The root's
//   min/max and select state come from one pass over all rows.
//   bottom levels: one 1024-thread CTA per segment finishes its whole subtree in
//     shared memory: nodes own aligned power-of-two slot blocks; per sub-level a
//     bitonic sort of each block by (value, pixel-index rank) puts the left child
//     first, then the right child moves to the block's second half.
#include "ff_internal.cuh"

namespace ff {

constexpr int SUB_MAX = 1024;  // largest segment finished by one CTA
constexpr int DIGIT = 12;
constexpr int NBINS = 1 << DIGIT;
constexpr int KD_CHUNK = 1024;      // positions per CTA of the top-level kernels (<= 2 segments)
// Longest collected list selected by a shared-memory sort, and the digit of the
// radix passes over longer lists. Both keep the collect kernel's shared memory
// small (about 5 KB), so that its CTAs do not crowd out the other streams' work.
constexpr int SEL_SORT_MAX = 512;
constexpr int SEL_DIGIT = 8;

int kd_depth(int N, int leaf) {
  int d = 0;
  while (((long long)N + (1ll << d) - 1) / (1ll << d) > leaf) d++;
  return d;
}

static int kd_top_levels(int N, int D) {
  int t = 0;
  while (((long long)N + (1ll << t) - 1) / (1ll << t) > SUB_MAX) t++;
  return t < D ? t : D;
}

__host__ __device__ static int bits_for(long long v) {  // bits to represent 0..v
  int b = 0;
  while ((1ll << b) <= v) b++;
  return b;
}

size_t kd_scratch_bytes(int N, int leaf) {
  KdBuild b{};
  b.N = N;
  b.leaf = leaf;
  Arena a;
  kd_bind_scratch(b, a);
  return a.off;
}

void kd_bind_scratch(KdBuild &b, Arena &a) {
  b.D = kd_depth(b.N, b.leaf);
  b.top_levels = kd_top_levels(b.N, b.D);
  int T = b.top_levels;
  int segs = 1 << (T > 0 ? T - 1 : 0);  // widest top level processed
  const size_t n1 = b.N > 0 ? b.N : 1;
  b.perm_tmp = a.take<int32_t>(n1);
  b.seg_off = a.take<int32_t>((size_t)(1 << (T + 1)) + T + 2);
  b.mm = a.take<int32_t>((size_t)2 * segs * NFEAT * 2);  // two levels (ping-pong)
  b.hist = a.take<uint32_t>((size_t)segs * NBINS);
  b.sel = a.take<int32_t>((size_t)2 * segs * 8);
  b.cnt = a.take<int32_t>((size_t)2 * segs * 2);
  b.ccnt = a.take<int32_t>((size_t)2 * segs);
  b.arrive = a.take<int32_t>((size_t)segs);
  b.keys = a.take<unsigned long long>(T > 0 ? n1 : 1);
  b.coll = a.take<unsigned long long>(T > 0 ? n1 : 1);
}

__host__ __device__ __forceinline__ int seg_base(int d) { return (1 << d) - 1 + d; }

// Levels ping-pong between perm and perm_tmp: level d reads cur_perm(d) and its
// partition writes cur_perm(d + 1).
__device__ __forceinline__ int32_t *cur_perm(const KdBuild &T, int d) {
  return (d & 1) ? T.perm_tmp : T.perm;
}
__device__ __forceinline__ int top_segs(const KdBuild &T) {
  return 1 << (T.top_levels > 0 ? T.top_levels - 1 : 0);
}
// Per-level state of segment s at level d: two buffers alternate by level parity.
__device__ __forceinline__ int32_t *mm_at(const KdBuild &T, int d, int s) {
  return T.mm + ((size_t)(d & 1) * top_segs(T) + s) * NFEAT * 2;
}
// select state: [0] dim, [1] vmin, [2] key bits B, [3] ibits, [4] remaining rank
// k, [5] prefix lo, [6] prefix hi, [7] bits consumed (B once the key is exact)
__device__ __forceinline__ int32_t *sel_at(const KdBuild &T, int d, int s) {
  return T.sel + ((size_t)(d & 1) * top_segs(T) + s) * 8;
}
__device__ __forceinline__ int32_t *cnt_at(const KdBuild &T, int d, int s) {
  return T.cnt + ((size_t)(d & 1) * top_segs(T) + s) * 2;
}
__device__ __forceinline__ int32_t *ccnt_at(const KdBuild &T, int d, int s) {
  return T.ccnt + (size_t)(d & 1) * top_segs(T) + s;
}
__device__ __forceinline__ unsigned long long sel_key(const int32_t *S) {
  return ((unsigned long long)(unsigned)S[6] << 32) | (unsigned)S[5];
}

__global__ void k_kd_seg_off(KdBuild *trees, int ntrees) {
  KdBuild &T = trees[blockIdx.y];
  for (int d = 0; d <= T.top_levels; d++) {
    int cnt = (1 << d) + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
      T.seg_off[seg_base(d) + i] = seg_begin(T.N, d, i);
  }
}

// Identity permutation; zero the radix histograms (each digit step clears the
// bins it used, so this is their only reset), the arrival counts, and the root's
// min/max sentinels.
__global__ void k_kd_init_perm(KdBuild *trees) {
  KdBuild &T = trees[blockIdx.y];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int i = tid; i < T.N; i += nth) T.perm[i] = i;
  if (T.top_levels > 0) {
    const int segs = top_segs(T);
    const size_t nbins = (size_t)segs * NBINS;
    for (size_t i = tid; i < nbins; i += nth) T.hist[i] = 0;
    for (int i = tid; i < segs; i += nth) T.arrive[i] = 0;
    for (int i = tid; i < NFEAT; i += nth) {
      int32_t *m = mm_at(T, 0, 0) + i * 2;
      m[0] = INT32_MAX;
      m[1] = INT32_MIN;
    }
  }
}

// Segment containing position pos at depth d (binary search in seg_off).
__device__ __forceinline__ int find_seg(const int32_t *off, int nseg, int pos) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= pos) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Select state of segment s at level d from its min/max (read through L2: other
// CTAs produced them), by one warp: lane k reads dimension k's min/max; the
// split dimension (largest max - min, lowest dimension on ties) by one warp max
// over the key (spread << 5) | (31 - lane). It also zeroes the segment's
// counters and, below the last top level, resets its children's min/max.
__device__ void seg_sel_init(KdBuild &T, int d, int s) {
  const int lane = threadIdx.x & 31;
  const int32_t *mm = mm_at(T, d, s);
  long long key = -1;
  if (lane < NFEAT) {
    const long long sp = (long long)__ldcg(mm + lane * 2 + 1) - __ldcg(mm + lane * 2);  // < 2^32
    if (sp >= 0) key = (sp << 5) | (31 - lane);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const long long y = __shfl_xor_sync(0xffffffffu, key, o);
    key = y > key ? y : key;
  }
  const int best = key >= 0 ? 31 - (int)(key & 31) : 0;
  const long long bs = key >= 0 ? key >> 5 : -1;
  if (lane == 0) {
    const int32_t *off = T.seg_off + seg_base(d);
    const int m = off[s + 1] - off[s];
    int vbits = bits_for(bs), ibits = bits_for(T.N - 1);
    if (ibits < 1) ibits = 1;
    int32_t *S = sel_at(T, d, s);
    S[0] = best;
    S[1] = __ldcg(mm + best * 2);
    S[2] = vbits + ibits;
    S[3] = ibits;
    S[4] = m / 2;
    S[5] = 0;
    S[6] = 0;
    S[7] = 0;
    T.split_dim[(1 << d) - 1 + s] = best;
    cnt_at(T, d, s)[0] = 0;
    cnt_at(T, d, s)[1] = 0;
    *ccnt_at(T, d, s) = 0;
  }
  if (d + 1 < T.top_levels && lane < NFEAT)
    for (int c = 0; c < 2; c++) {
      int32_t *m = mm_at(T, d + 1, 2 * s + c);
      m[2 * lane] = INT32_MAX;
      m[2 * lane + 1] = INT32_MIN;
    }
}

// Arrival bookkeeping of a chunk CTA at level d: after the CTA's global updates
// for the segments [seg0, seg_of(end - 1)] it touched, one fence and one
// increment per segment; returns the mask (bit i: segment seg0 + i) of segments
// whose last chunk this CTA was, their counts reset for the next kernel. Every
// thread of the CTA must call it. Nothing waits: the CTA that completes a
// segment sees every other chunk's updates through the fences.
__device__ __forceinline__ int chunks_of(const int32_t *off, int s) {
  const int b = off[s], e = off[s + 1];
  return e > b ? (e - 1) / KD_CHUNK - b / KD_CHUNK + 1 : 0;
}
__device__ unsigned finish_chunk(KdBuild &T, const int32_t *off, int nseg, int end, int seg0) {
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned last = 0;
    const int s1 = find_seg(off, nseg, end - 1);
    for (int sg = seg0; sg <= s1 && sg - seg0 < 32; sg++) {
      if (atomicAdd(&T.arrive[sg], 1) == chunks_of(off, sg) - 1) {
        last |= 1u << (sg - seg0);
        T.arrive[sg] = 0;
      }
    }
    s_last = last;
  }
  __syncthreads();
  const unsigned last = s_last;
  if (last) __threadfence();
  return last;
}

// Per-dimension min/max of the root (all N feature rows): the rows are read in
// memory order, each warp walks a strided set of rows with lanes = dimensions
// and four rows in flight, then warp results merge in shared memory and once per
// CTA in global memory. The last CTA of a tree sets up the root's select state.
constexpr int MM_ROWS_PER_WARP = 64;

__global__ void __launch_bounds__(256) k_kd_minmax_root(KdBuild *trees) {
  KdBuild &T = trees[blockIdx.y];
  if (T.top_levels <= 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = (blockIdx.x * 8 + warp) * MM_ROWS_PER_WARP;
  __shared__ int smin[NFEAT], smax[NFEAT];
  __shared__ int s_last;
  if (tid < NFEAT) {
    smin[tid] = INT32_MAX;
    smax[tid] = INT32_MIN;
  }
  __syncthreads();
  if (r0 < T.N && lane < NFEAT) {
    const int r1 = min(r0 + MM_ROWS_PER_WARP, T.N);
    int lo = INT32_MAX, hi = INT32_MIN;
    if (T.packed) {
      const uint32_t *rows = (const uint32_t *)T.feat;
#pragma unroll 4
      for (int r = r0; r < r1; r++) {
        const int v = packed_feat_value(rows + (size_t)r * FEAT_PACKED_WORDS, lane);
        lo = min(lo, v);
        hi = max(hi, v);
      }
    } else {
      const int32_t *col = T.feat + lane;
#pragma unroll 4
      for (int r = r0; r < r1; r++) {
        const int v = col[(size_t)r * FEAT_STRIDE];
        lo = min(lo, v);
        hi = max(hi, v);
      }
    }
    atomicMin(&smin[lane], lo);
    atomicMax(&smax[lane], hi);
  }
  __syncthreads();
  if (tid < NFEAT && smin[tid] != INT32_MAX) {
    atomicMin(&mm_at(T, 0, 0)[tid * 2], smin[tid]);
    atomicMax(&mm_at(T, 0, 0)[tid * 2 + 1], smax[tid]);
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    s_last = atomicAdd(&T.arrive[0], 1) == (int)gridDim.x - 1;
    if (s_last) T.arrive[0] = 0;
  }
  __syncthreads();
  if (s_last && warp == 0) {
    __threadfence();
    seg_sel_init(T, 0, 0);
  }
}

// Feature value / whole row of point idx in either row layout.
__device__ __forceinline__ int feat_value(const KdBuild &T, int idx, int dim) {
  return T.packed ? packed_feat_value((const uint32_t *)T.feat + (size_t)idx * FEAT_PACKED_WORDS, dim)
                  : T.feat[(size_t)idx * FEAT_STRIDE + dim];
}
template <bool PACKED>
__device__ __forceinline__ void feat_row_as(const KdBuild &T, int idx, bool ok, int32_t *v) {
  if (PACKED) {
    uint4 q[4];
    const uint4 *row = (const uint4 *)((const uint32_t *)T.feat + (size_t)idx * FEAT_PACKED_WORDS);
#pragma unroll
    for (int k = 0; k < 4; k++) q[k] = ok ? row[k] : make_uint4(0, 0, 0, 0);
    unpack_feat_row((const uint32_t *)q, v);
  } else {
    int4 q[7];
    const int4 *row = (const int4 *)(T.feat + (size_t)idx * FEAT_STRIDE);
#pragma unroll
    for (int k = 0; k < 7; k++) q[k] = ok ? row[k] : make_int4(0, 0, 0, 0);
#pragma unroll
    for (int k = 0; k < NFEAT; k++) v[k] = ((const int *)q)[k];
  }
}
__device__ __forceinline__ void feat_row(const KdBuild &T, int idx, bool ok, int32_t *v) {
  if (T.packed) feat_row_as<true>(T, idx, ok, v);
  else feat_row_as<false>(T, idx, ok, v);
}

__device__ __forceinline__ unsigned long long kd_key(const KdBuild &T, const int32_t *S, int idx) {
  int v = feat_value(T, idx, S[0]);
  return ((unsigned long long)(unsigned)(v - S[1]) << S[3]) | (unsigned)idx;
}

constexpr int CHUNK_SEGS = 4;  // segment slots per chunk

// The segments a chunk of positions touches (top levels: at most CHUNK_SEGS):
// first segment and the begin offsets of the following ones, in shared memory.
__device__ __forceinline__ void chunk_segments(const int32_t *off, int nseg, int start, int *sseg0,
                                               int *sbound) {
  if (threadIdx.x == 0) {
    const int s0 = find_seg(off, nseg, start);
    *sseg0 = s0;
    for (int i = 0; i < CHUNK_SEGS - 1; i++) sbound[i] = s0 + 1 + i <= nseg ? off[s0 + 1 + i] : INT32_MAX;
  }
}
__device__ __forceinline__ int seg_of(int p, int seg0, const int *sbound) {
  int s = seg0;
#pragma unroll
  for (int i = 0; i < CHUNK_SEGS - 1; i++) s += p >= sbound[i];
  return s;
}

// Digit step of segment s at level d (its histogram complete, read through L2):
// the bin holding rank k, the narrowed prefix, the bins cleared for the next
// level. Run by all 256 threads of one CTA.
__device__ void seg_digit(KdBuild &T, int d, int s) {
  int32_t *S = sel_at(T, d, s);
  const int B = S[2], used = S[7];
  uint32_t *h = T.hist + (size_t)s * NBINS;
  if (used >= B) return;  // uniform
  const int hi = B - used, lo = max(hi - DIGIT, 0), nb = 1 << (hi - lo);
  __shared__ uint32_t part[256];
  __shared__ int found_bin, found_before, s_tt;
  __shared__ uint32_t s_before;
  // each thread holds a run of NBINS / 256 consecutive bins in registers (four
  // 16-byte loads) and sums it
  constexpr int per = NBINS / 256;
  uint32_t v[per];
  {
    const uint4 *h4 = (const uint4 *)(h + threadIdx.x * per);
#pragma unroll
    for (int q = 0; q < per / 4; q++) {
      const uint4 x = __ldcg(h4 + q);
      v[4 * q] = x.x;
      v[4 * q + 1] = x.y;
      v[4 * q + 2] = x.z;
      v[4 * q + 3] = x.w;
    }
  }
  uint32_t mine = 0;
#pragma unroll
  for (int i = 0; i < per; i++) {
    if ((int)threadIdx.x * per + i >= nb) v[i] = 0;
    mine += v[i];
  }
  part[threadIdx.x] = mine;
  __syncthreads();
  const uint32_t k = (uint32_t)S[4];
  // the run holding rank k: inclusive prefix sums of the 256 runs by warp 0 (8
  // runs per lane)
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    uint32_t w[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) sum += (w[i] = part[lane * 8 + i]);
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t acc = incl - sum;  // runs before this lane's eight
    int t = -1;
    uint32_t before = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      if (t < 0 && acc + w[i] > k) {
        t = lane * 8 + i;
        before = acc;
      }
      acc += w[i];
    }
    const unsigned hit = __ballot_sync(0xffffffffu, t >= 0);
    const int src = hit ? __ffs(hit) - 1 : 31;
    int tt = __shfl_sync(0xffffffffu, t, src);
    before = __shfl_sync(0xffffffffu, before, src);
    const uint32_t last = __shfl_sync(0xffffffffu, w[7], 31), total = __shfl_sync(0xffffffffu, incl, 31);
    if (!hit) {  // rank beyond the total: the last run, as a sequential scan would stop
      tt = 255;
      before = total - last;
    }
    if (lane == 0) {
      s_tt = tt;
      s_before = before;
    }
  }
  __syncthreads();
  // the run's owner finds the bin inside it from its registers: advance while the
  // bin still lies before rank k (at most per - 1 bins)
  if ((int)threadIdx.x == s_tt) {
    uint32_t a2 = s_before;
    int at = per - 1;
    bool stop = false;
#pragma unroll
    for (int i = 0; i < per - 1; i++) {
      if (!stop) {
        if (a2 + v[i] <= k) {
          a2 += v[i];
        } else {
          at = i;
          stop = true;
        }
      }
    }
    found_bin = s_tt * per + at;
    found_before = (int)a2;
  }
  __syncthreads();
  {  // each thread clears the run it read
    uint4 *h4 = (uint4 *)(h + threadIdx.x * per);
#pragma unroll
    for (int q = 0; q < per / 4; q++) h4[q] = make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x == 0) {
    unsigned long long pre = sel_key(S);
    pre = (pre << (hi - lo)) | (unsigned)found_bin;
    S[5] = (int32_t)(pre & 0xffffffffu);
    S[6] = (int32_t)(pre >> 32);
    S[4] -= found_before;
    S[7] = used + (hi - lo);
  }
  __syncthreads();
}

// Level d's radix pass over the top digit: every position's key (gathered from
// its feature row, cached in T.keys) counted in its segment's histogram; the last
// chunk of a segment runs its digit step.
__global__ void __launch_bounds__(256, 5) k_kd_hist(KdBuild *trees, int d) {
  KdBuild &T = trees[blockIdx.y];
  if (d >= T.top_levels) return;
  const int start = blockIdx.x * KD_CHUNK;
  if (start >= T.N) return;
  const int end = min(start + KD_CHUNK, T.N);
  const int nseg = 1 << d;
  const int32_t *off = T.seg_off + seg_base(d);
  __shared__ uint32_t sh[NBINS];
  __shared__ int sseg0, sbound[CHUNK_SEGS - 1];
  chunk_segments(off, nseg, start, &sseg0, sbound);
  for (int i = threadIdx.x; i < NBINS; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int seg0 = sseg0;
  const bool single = sbound[0] >= end;
  for (int p = start + threadIdx.x; p < end; p += blockDim.x) {
    const int s = single ? seg0 : seg_of(p, seg0, sbound);
    const int32_t *S = sel_at(T, d, s);
    const int B = S[2], lo = max(B - DIGIT, 0);
    const unsigned long long K = kd_key(T, S, cur_perm(T, d)[p]);
    T.keys[p] = K;
    const unsigned dig = (unsigned)((K >> lo) & ((1ull << (B - lo)) - 1));
    if (single) atomicAdd(&sh[dig], 1u);
    else atomicAdd(&T.hist[(size_t)s * NBINS + dig], 1u);
  }
  __syncthreads();
  if (single)
    for (int i = threadIdx.x; i < NBINS; i += blockDim.x)
      if (sh[i]) atomicAdd(&T.hist[(size_t)seg0 * NBINS + i], sh[i]);
  const unsigned last = finish_chunk(T, off, nseg, end, seg0);
  for (int i = 0; i < CHUNK_SEGS; i++)
    if (last & (1u << i)) seg_digit(T, d, seg0 + i);
}

// Exact key of the remaining rank S[4] among segment s's collected keys (the
// bucket of the top digit), by all 256 threads of one CTA: a bitonic sort in
// shared memory for lists of up to SEL_SORT_MAX keys, else radix passes of
// SEL_DIGIT bits over the list in global memory. The result becomes the selected
// key.
__device__ void seg_select(KdBuild &T, int d, int s) {
  int32_t *S = sel_at(T, d, s);
  const int B = S[2];
  if (S[7] >= B) return;  // uniform: the top digit already fixed the key
  const int32_t *off = T.seg_off + seg_base(d);
  const int c = min(__ldcg(ccnt_at(T, d, s)), off[s + 1] - off[s]);  // the list fits its segment
  const unsigned long long *list = T.coll + off[s];
  const int tid = threadIdx.x;
  __shared__ unsigned long long sk[SEL_SORT_MAX];
  __shared__ unsigned long long s_key, s_pre;
  __shared__ uint32_t hs[1 << SEL_DIGIT];
  __shared__ uint32_t s_k;
  __shared__ int s_used;
  const uint32_t k0 = (uint32_t)S[4];
  if (c <= SEL_SORT_MAX) {
    int n2 = 1;
    while (n2 < c) n2 <<= 1;
    for (int i = tid; i < n2; i += blockDim.x) sk[i] = i < c ? __ldcg(list + i) : ~0ull;
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < n2; i += blockDim.x) {
          const int ij = i ^ j;
          if (ij > i) {
            const unsigned long long a = sk[i], b = sk[ij];
            if ((a > b) == ((i & k) == 0)) {
              sk[i] = b;
              sk[ij] = a;
            }
          }
        }
        __syncthreads();
      }
    if (tid == 0) s_key = sk[k0 < (uint32_t)c ? k0 : (uint32_t)(c > 0 ? c - 1 : 0)];
  } else {
    if (tid == 0) {
      s_pre = sel_key(S);
      s_k = k0;
      s_used = S[7];
    }
    __syncthreads();
    while (s_used < B) {  // s_used is shared: the loop is uniform
      const int hi = B - s_used, lo = max(hi - SEL_DIGIT, 0), nb = 1 << (hi - lo);
      const unsigned long long pre = s_pre;
      for (int i = tid; i < (1 << SEL_DIGIT); i += blockDim.x) hs[i] = 0;
      __syncthreads();
      for (int i = tid; i < c; i += blockDim.x) {
        const unsigned long long K = __ldcg(list + i);
        if ((K >> hi) == pre) atomicAdd(&hs[(unsigned)((K >> lo) & (unsigned long long)(nb - 1))], 1u);
      }
      __syncthreads();
      if (tid == 0) {  // the bin holding rank s_k
        uint32_t acc = 0;
        int bin = nb - 1;
        for (int i = 0; i < nb; i++) {
          if (acc + hs[i] > s_k) {
            bin = i;
            break;
          }
          acc += hs[i];
        }
        s_pre = (pre << (hi - lo)) | (unsigned)bin;
        s_k -= acc;
        s_used += hi - lo;
      }
      __syncthreads();
    }
    if (tid == 0) s_key = s_pre;
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned long long key = s_key;
    S[5] = (int32_t)(key & 0xffffffffu);
    S[6] = (int32_t)(key >> 32);
    S[4] = 0;
    S[7] = B;
  }
  __syncthreads();
}

// Collect: the cached keys that fall in the bin the top digit chose are appended
// to their segment's list; the last chunk of a segment selects its exact median
// key from the list.
__global__ void __launch_bounds__(256) k_kd_collect(KdBuild *trees, int d) {
  KdBuild &T = trees[blockIdx.y];
  if (d >= T.top_levels) return;
  const int start = blockIdx.x * KD_CHUNK;
  if (start >= T.N) return;
  const int end = min(start + KD_CHUNK, T.N);
  const int nseg = 1 << d;
  const int32_t *off = T.seg_off + seg_base(d);
  __shared__ int sseg0, sbound[CHUNK_SEGS - 1];
  chunk_segments(off, nseg, start, &sseg0, sbound);
  __syncthreads();
  const int seg0 = sseg0;
  for (int p = start + threadIdx.x; p < end; p += blockDim.x) {
    const int s = seg_of(p, seg0, sbound);
    const int32_t *S = sel_at(T, d, s);
    const int B = S[2], used = S[7];
    if (used >= B) continue;
    const unsigned long long K = T.keys[p];
    if ((K >> (B - used)) == sel_key(S)) {
      const int slot = atomicAdd(ccnt_at(T, d, s), 1);
      if (slot < off[s + 1] - off[s]) T.coll[off[s] + slot] = K;
      else raise_status(T.status, DEV_ERR_KD, s, d);
    }
  }
  const unsigned last = finish_chunk(T, off, nseg, end, seg0);
  for (int i = 0; i < CHUNK_SEGS; i++)
    if (last & (1u << i)) seg_select(T, d, seg0 + i);
}

// Partition: key < selected key goes to the left child, else right. Positions
// come from per-segment counters, aggregated per warp (match_any on the
// destination) and per CTA, so a CTA issues at most one global atomic per
// destination child (order inside a child is unspecified). The selected point
// writes the split value. While the rows pass through, the per-dimension
// min/max of the children (next level) is accumulated per child present in the
// warp: one child at a time, all lanes converged, full-mask warp reductions in
// which the other lanes contribute the neutral value, then shared and global
// atomics. The last chunk of a segment sets up its two children's select state
// for the next level. Rows are read in either layout (int32 or packed).
constexpr int PART_ROUNDS = KD_CHUNK / 256;

template <bool PACKED>
__global__ void __launch_bounds__(256, 5) k_kd_partition(KdBuild *trees, int d) {
  KdBuild &T = trees[blockIdx.y];
  if (d >= T.top_levels) return;
  const int start = blockIdx.x * KD_CHUNK;
  if (start >= T.N) return;
  const int end = min(start + KD_CHUNK, T.N);
  const int nseg = 1 << d;
  const int32_t *off = T.seg_off + seg_base(d);
  const int32_t *src = cur_perm(T, d);
  int32_t *dstp = cur_perm(T, d + 1);
  const bool child_mm = d + 1 < T.top_levels;
  __shared__ int s_seg0, s_bound[CHUNK_SEGS - 1];
  __shared__ int s_cnt[8], s_base[8];
  __shared__ int s_min[8][NFEAT], s_max[8][NFEAT];
  const int tid = threadIdx.x, lane = tid & 31;
  chunk_segments(off, nseg, start, &s_seg0, s_bound);
  if (tid < 8) s_cnt[tid] = 0;
  for (int i = tid; i < 8 * NFEAT; i += 256) {
    s_min[i / NFEAT][i % NFEAT] = INT32_MAX;
    s_max[i / NFEAT][i % NFEAT] = INT32_MIN;
  }
  __syncthreads();
  const int seg0 = s_seg0;
  int combo[PART_ROUNDS], rank[PART_ROUNDS], idxs[PART_ROUNDS];
#pragma unroll
  for (int r = 0; r < PART_ROUNDS; r++) {
    const int p = start + r * 256 + tid;
    int c = -1, idx = 0;
    if (p < end) {
      const int sg = seg_of(p, seg0, s_bound);
      const int32_t *S = sel_at(T, d, sg);
      idx = src[p];
      const unsigned long long K = T.keys[p];  // cached by the level's histogram pass
      const unsigned long long sel = sel_key(S);
      c = 2 * (sg - seg0) + (K < sel ? 0 : 1);
      if (K == sel) T.split_val[(1 << d) - 1 + sg] = (int)(K >> S[3]) + S[1];
    }
    const unsigned grp = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(grp) - 1;
    int wbase = 0;
    if (c >= 0 && lane == leader) wbase = atomicAdd(&s_cnt[c], __popc(grp));
    wbase = __shfl_sync(0xffffffffu, wbase, leader);
    combo[r] = c;
    rank[r] = wbase + __popc(grp & ((1u << lane) - 1));
    idxs[r] = idx;
    if (child_mm) {  // child min/max over the full rows
      int32_t v[NFEAT];
      feat_row_as<PACKED>(T, idx, c >= 0, v);
      // one child slot at a time, all lanes converged, full-mask reductions in
      // which the other lanes contribute the neutral value
      unsigned todo = __ballot_sync(0xffffffffu, c >= 0);
      while (todo) {
        const int lead = __ffs(todo) - 1;
        const int cc = __shfl_sync(0xffffffffu, c, lead);
        const bool mine = c == cc;
        todo &= ~__ballot_sync(0xffffffffu, mine);
#pragma unroll
        for (int dim = 0; dim < NFEAT; dim++) {
          const int lo = __reduce_min_sync(0xffffffffu, mine ? v[dim] : INT32_MAX);
          const int hi = __reduce_max_sync(0xffffffffu, mine ? v[dim] : INT32_MIN);
          if (lane == lead) {
            atomicMin(&s_min[cc][dim], lo);
            atomicMax(&s_max[cc][dim], hi);
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid < 8 && s_cnt[tid] > 0 && seg0 + (tid >> 1) < nseg)
    s_base[tid] = atomicAdd(&cnt_at(T, d, seg0 + (tid >> 1))[tid & 1], s_cnt[tid]);
  if (child_mm)
    for (int i = tid; i < 8 * NFEAT; i += 256) {
      const int c = i / NFEAT, dim = i % NFEAT;
      if (s_min[c][dim] == INT32_MAX) continue;
      int32_t *m = mm_at(T, d + 1, 2 * (seg0 + (c >> 1)) + (c & 1));
      atomicMin(&m[dim * 2], s_min[c][dim]);
      atomicMax(&m[dim * 2 + 1], s_max[c][dim]);
    }
  __syncthreads();
  if (child_mm) {  // before the scatter: the fence then covers only the atomics above
    const unsigned last = finish_chunk(T, off, nseg, end, seg0);
    // warps 2i and 2i + 1 set up the two children of the i-th completed segment
    const int warp = tid >> 5;
    if (warp < 2 * CHUNK_SEGS && (last & (1u << (warp >> 1))))
      seg_sel_init(T, d + 1, 2 * (seg0 + (warp >> 1)) + (warp & 1));
  }
#pragma unroll
  for (int r = 0; r < PART_ROUNDS; r++) {
    const int c = combo[r];
    if (c < 0) continue;
    const int sg = seg0 + (c >> 1), side = c & 1;
    const int b = off[sg], m = off[sg + 1] - b, half = m >> 1;
    const int k = s_base[c] + rank[r];
    const int lim = side ? m - half : half;
    if (k < lim) dstp[b + side * half + k] = idxs[r];
    else raise_status(T.status, DEV_ERR_KD, sg, d);
  }
}

// Ascending bitonic sort of one 64-bit key per thread within aligned blocks of
// B threads (B a power of two, 2..SUB_MAX): thread t ends with the (t mod B)-th
// smallest key of its block. Exchanges with partners inside the warp use
// shuffles; wider ones go through shared memory (two buffers, so one barrier per
// step suffices). Every thread of the CTA must call it with the same B.
__device__ __forceinline__ unsigned long long bitonic_sort_blocks(unsigned long long c, int B,
                                                                  unsigned long long *buf) {
  const int t = threadIdx.x;
  int flip = 0;
  for (int k = 2; k <= B; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      unsigned long long o;
      if (j >= 32) {
        unsigned long long *b = buf + flip * SUB_MAX;
        b[t] = c;
        __syncthreads();
        o = b[t ^ j];
        flip ^= 1;
      } else {
        o = __shfl_xor_sync(0xffffffffu, c, j);
      }
      const bool up = (k == B) || ((t & k) == 0), lower = (t & j) == 0;
      c = (lower == up) ? (o < c ? o : c) : (o > c ? o : c);
    }
  }
  return c;
}

// The same for 32-bit keys (one shuffle per exchange).
__device__ __forceinline__ uint32_t bitonic_sort_blocks32(uint32_t c, int B, uint32_t *buf) {
  const int t = threadIdx.x;
  int flip = 0;
  for (int k = 2; k <= B; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      uint32_t o;
      if (j >= 32) {
        uint32_t *b = buf + flip * SUB_MAX;
        b[t] = c;
        __syncthreads();
        o = b[t ^ j];
        flip ^= 1;
      } else {
        o = __shfl_xor_sync(0xffffffffu, c, j);
      }
      const bool up = (k == B) || ((t & k) == 0), lower = (t & j) == 0;
      c = (lower == up) ? min(o, c) : max(o, c);
    }
  }
  return c;
}

// One 1024-thread CTA finishes the subtree of one segment at depth top_levels.
// The segment's points live in shared memory with their 27 features; at
// sub-level sd node j owns the aligned slot block [j B, j B + B), B = 1024 >> sd,
// its m_j points first. Per sub-level: per-node min/max of every dimension
// (segmented warp reductions, then across the node's warps), the split
// dimension, a bitonic sort of each block by (value - node min, pixel-index
// rank, slot), and one move of every point to its child's block: the first
// floor(m/2) stay, the others go to the second half. The first point of the
// right half is the split. The pixel-index rank (0..1023) breaks ties exactly as
// the pixel index does; it is set once by sorting the segment's indices. When
// every node's spread in its split dimension is below 2^21 (always for WHT
// features, |value| <= 289 * 255) the sort key is the 32-bit (value - node min,
// rank) and a rank -> slot table finds each key's point; otherwise the 64-bit
// key carries the slot itself.
constexpr int SUB_SD_SMEM_NODES = SUB_MAX / 64;  // nodes with blocks wider than a warp

__global__ void __launch_bounds__(SUB_MAX) k_kd_subtree(KdBuild *trees) {
  KdBuild &T = trees[blockIdx.y];
  const int d0 = T.top_levels;
  if (blockIdx.x >= (1u << d0)) return;
  const int b0 = seg_begin(T.N, d0, blockIdx.x), e0 = seg_begin(T.N, d0, blockIdx.x + 1);
  const int m0 = e0 - b0;
  extern __shared__ __align__(16) int32_t ssub[];
  unsigned long long *sbuf = (unsigned long long *)ssub;  // 2 x SUB_MAX sort buffers
  int32_t *ssorted = (int32_t *)(sbuf + 2 * SUB_MAX);      // SUB_MAX: source slot of sorted key
  int32_t *sslot = ssorted + SUB_MAX;                      // SUB_MAX: slot of each rank
  int32_t *sF = sslot + SUB_MAX;                           // SUB_MAX x NFEAT features
  int32_t *sidx = sF + SUB_MAX * NFEAT;                    // pixel index per slot
  int32_t *srank = sidx + SUB_MAX;                         // pixel-index rank per slot
  int32_t *ssize = srank + SUB_MAX;                        // 2 x SUB_MAX node sizes (ping-pong)
  int32_t *sstart = ssize + 2 * SUB_MAX;                   // 2 x SUB_MAX node starts
  int32_t *smin = sstart + 2 * SUB_MAX;                    // SUB_SD_SMEM_NODES x NFEAT
  int32_t *smax = smin + SUB_SD_SMEM_NODES * NFEAT;
  int32_t *swmin = smax + SUB_SD_SMEM_NODES * NFEAT;       // per warp x NFEAT
  int32_t *swmax = swmin + (SUB_MAX / 32) * NFEAT;
  int32_t *sdim = swmax + (SUB_MAX / 32) * NFEAT;          // SUB_SD_SMEM_NODES
  int32_t *sdmin = sdim + SUB_SD_SMEM_NODES;
  const int t = threadIdx.x, lane = t & 31;
  // slots in pixel-index order: slot t holds the t-th smallest index, rank t
  {
    const uint32_t raw = t < m0 ? (uint32_t)cur_perm(T, d0)[b0 + t] : 0xffffffffu;  // idx < 2^31
    const uint32_t srt = bitonic_sort_blocks32(raw, SUB_MAX, (uint32_t *)sbuf);
    if (t < m0) {
      const int idx = (int)srt;
      sidx[t] = idx;
      srank[t] = t;
      sslot[t] = t;
      int32_t v[NFEAT];
      feat_row(T, idx, true, v);
#pragma unroll
      for (int k = 0; k < NFEAT; k++) sF[t * NFEAT + k] = v[k];
    }
    if (t == 0) {
      ssize[0] = m0;
      sstart[0] = 0;
    }
  }
  const int levels = T.D - d0;
  int pp = 0;  // ping-pong half of the node arrays
  for (int sd = 0; sd < levels; sd++) {
    const int B = SUB_MAX >> sd, j = t / B, o = t & (B - 1);
    __syncthreads();
    const int m = ssize[pp * SUB_MAX + j], st = sstart[pp * SUB_MAX + j];
    const bool valid = o < m;
    // per-node min/max of every dimension and the split dimension (largest
    // max - min, lowest dimension on ties)
    int dim = 0, dmin = 0;
    if (B <= 32) {  // the node is a segment of a warp: reductions in registers
      const unsigned bmask = B == 32 ? 0xffffffffu : (((1u << B) - 1u) << (lane & ~(B - 1)));
      long long best = -1;
#pragma unroll 9
      for (int k = 0; k < NFEAT; k++) {
        const int v = valid ? sF[t * NFEAT + k] : 0;
        const int lo = __reduce_min_sync(bmask, valid ? v : INT32_MAX);
        const int hi = __reduce_max_sync(bmask, valid ? v : INT32_MIN);
        if (m > 0 && (long long)hi - lo > best) {
          best = (long long)hi - lo;
          dim = k;
          dmin = lo;
        }
      }
    } else {  // per-warp results, then one thread per (node, dimension), then per node
      const int warp = t >> 5;
#pragma unroll 9
      for (int k = 0; k < NFEAT; k++) {
        const int v = valid ? sF[t * NFEAT + k] : 0;
        const int lo = __reduce_min_sync(0xffffffffu, valid ? v : INT32_MAX);
        const int hi = __reduce_max_sync(0xffffffffu, valid ? v : INT32_MIN);
        if (lane == 0) {
          swmin[warp * NFEAT + k] = lo;
          swmax[warp * NFEAT + k] = hi;
        }
      }
      __syncthreads();
      const int nn = SUB_MAX / B, wpn = B / 32;
      if (t < nn * NFEAT) {
        const int node = t / NFEAT, k = t % NFEAT;
        int lo = INT32_MAX, hi = INT32_MIN;
        for (int w = node * wpn; w < (node + 1) * wpn; w++) {
          lo = min(lo, swmin[w * NFEAT + k]);
          hi = max(hi, swmax[w * NFEAT + k]);
        }
        smin[t] = lo;
        smax[t] = hi;
      }
      __syncthreads();
      if (t < nn) {
        long long best = -1;
        int bd = 0, bm = 0;
        for (int k = 0; k < NFEAT; k++) {
          const long long sp = (long long)smax[t * NFEAT + k] - smin[t * NFEAT + k];
          if (sp > best) {
            best = sp;
            bd = k;
            bm = smin[t * NFEAT + k];
          }
        }
        sdim[t] = bd;
        sdmin[t] = bm;
      }
      __syncthreads();
      dim = sdim[j];
      dmin = sdmin[j];
    }
    const uint32_t vrel = valid ? (uint32_t)(sF[t * NFEAT + dim] - dmin) : 0u;
    if (__syncthreads_or(vrel >= (1u << 21)) == 0) {  // valid keys < 2^31: never the sentinel
      const uint32_t key = valid ? (vrel << 10) | (uint32_t)srank[t] : 0xffffffffu;
      const uint32_t sorted = bitonic_sort_blocks32(key, B, (uint32_t *)sbuf);
      ssorted[t] = sorted == 0xffffffffu ? 0 : sslot[sorted & 1023u];
    } else {
      const unsigned long long key =
          valid ? ((unsigned long long)vrel << 20) | ((unsigned long long)srank[t] << 10) | (unsigned)t
                : ~0ull;
      const unsigned long long sorted = bitonic_sort_blocks(key, B, sbuf);
      ssorted[t] = (int)(sorted & 1023u);
    }
    __syncthreads();
    // move: the first floor(m/2) stay at the front of the block, the others go
    // to the front of its second half
    const int h = m >> 1, half = B >> 1;
    const int sp = o < half ? o : h + (o - half);
    const bool take = o < half ? o < h : sp < m;
    int32_t f[NFEAT];
    int pidx = 0, prank = 0;
    if (take) {
      const int src = ssorted[j * B + sp];
#pragma unroll
      for (int k = 0; k < NFEAT; k++) f[k] = sF[src * NFEAT + k];
      pidx = sidx[src];
      prank = srank[src];
    }
    __syncthreads();
    if (take) {
#pragma unroll
      for (int k = 0; k < NFEAT; k++) sF[t * NFEAT + k] = f[k];
      sidx[t] = pidx;
      srank[t] = prank;
      sslot[prank] = t;
      if (o == half) {  // the first point of the right child is the split
        const int node = (1 << (d0 + sd)) - 1 + (blockIdx.x << sd) + j;
        T.split_dim[node] = dim;
        int sv = 0;
#pragma unroll
        for (int k = 0; k < NFEAT; k++)
          if (k == dim) sv = f[k];
        T.split_val[node] = sv;
      }
    }
    if (o == 0) {
      const int q = (pp ^ 1) * SUB_MAX + 2 * j;
      ssize[q] = h;
      ssize[q + 1] = m - h;
      sstart[q] = st;
      sstart[q + 1] = st + h;
    }
    pp ^= 1;
  }
  __syncthreads();
  {
    const int B = SUB_MAX >> levels, j = t / B, o = t & (B - 1);
    if (o < ssize[pp * SUB_MAX + j]) T.perm[b0 + sstart[pp * SUB_MAX + j] + o] = sidx[t];
  }
}

static size_t subtree_smem() {
  return sizeof(unsigned long long) * 2 * SUB_MAX +
         sizeof(int32_t) * ((size_t)SUB_MAX * NFEAT + 8 * SUB_MAX + 2 * SUB_SD_SMEM_NODES * NFEAT +
                            2 * (SUB_MAX / 32) * NFEAT + 2 * SUB_SD_SMEM_NODES);
}

ff_status launch_kd_build(const KdBuild *trees, KdBuild *dev, int ntrees, cudaStream_t st) {
  if (ntrees <= 0) return FF_OK;
  FF_TRY(upload_desc(trees, dev, ntrees, st));
  int maxT = 0, maxN = 0, maxSub = 0;
  for (int i = 0; i < ntrees; i++) {
    maxT = max(maxT, trees[i].top_levels);
    maxN = max(maxN, trees[i].N);
    maxSub = max(maxSub, trees[i].D - trees[i].top_levels);
  }
  if (maxN <= 0) return FF_OK;
  const bool packed = trees[0].packed != 0;  // one row layout per launch
  for (int i = 1; i < ntrees; i++)
    if ((trees[i].packed != 0) != packed) return FF_ERR_INVALID_ARG;
  const int B = 256;
  const int gN = min((maxN + B - 1) / B, 4096);
  k_kd_init_perm<<<dim3(gN, ntrees), B, 0, st>>>(dev);
  FF_CHECK_LAUNCH();
  k_kd_seg_off<<<dim3(8, ntrees), B, 0, st>>>(dev, ntrees);
  FF_CHECK_LAUNCH();
  // three launches per top level; the last chunk CTA of each segment chains the
  // segment's next step (digit, select, children's split dimension)
  const int chunks = (maxN + KD_CHUNK - 1) / KD_CHUNK;
  for (int d = 0; d < maxT; d++) {
    if (d == 0) {
      const int rows_per_cta = 8 * MM_ROWS_PER_WARP;
      k_kd_minmax_root<<<dim3((maxN + rows_per_cta - 1) / rows_per_cta, ntrees), 256, 0, st>>>(dev);
      FF_CHECK_LAUNCH();
    }
    k_kd_hist<<<dim3(chunks, ntrees), 256, 0, st>>>(dev, d);
    FF_CHECK_LAUNCH();
    k_kd_collect<<<dim3(chunks, ntrees), 256, 0, st>>>(dev, d);
    FF_CHECK_LAUNCH();
    if (packed)
      k_kd_partition<true><<<dim3(chunks, ntrees), 256, 0, st>>>(dev, d);
    else
      k_kd_partition<false><<<dim3(chunks, ntrees), 256, 0, st>>>(dev, d);
    FF_CHECK_LAUNCH();
  }
  if (maxSub > 10) return FF_ERR_INVALID_ARG;  // segments <= SUB_MAX points, leaf >= 1
  const size_t smem = subtree_smem();
  FF_TRY(smem_opt_in((const void *)k_kd_subtree, smem));
  k_kd_subtree<<<dim3(1 << maxT, ntrees), SUB_MAX, smem, st>>>(dev);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

// ---------------------------------------------------------------------------
// Eq. 1 / Eq. 4: per coarsest grid point, descend the tree with the point's WHT
// vector (left iff value < split value, no backtracking), then rerank the leaf's
// pixels by E_d on P^n_r: smallest cost wins, ties to the lowest pixel index.
// Then the K proposals in order, each replacing only with strictly lower cost.
// One half warp per grid point; lane 0 descends, the 16 lanes share each E_d.
// The tree may come from the caller (ff_kdtree_init): a split dimension outside
// [0, 27) or a leaf entry outside [0, N) is not dereferenced; it raises
// DEV_ERR_BOUNDS (grid point, node or position) and the descent takes dimension 0
// / the candidate is skipped.
template <int R>
__global__ void __launch_bounds__(256) k_kd_query(const KdQuery *qs) {
  const KdQuery &Q = qs[blockIdx.y];
  const int NX = Q.src.NX, G = NX * Q.src.NY, n = Q.src.n, W = Q.src.W;
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int l16 = threadIdx.x & 15;
  const unsigned gmask = 0xffffu << (threadIdx.x & 16);
  if (g >= G) return;  // uniform per half warp
  const int px = (g % NX) * n, py = (g / NX) * n;
  int leaf = 0;
  if (l16 == 0) {
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
  const uint32_t *sc = plane_centre(Q.src, px, py);
  int best = COST_UNSET, bidx = 0x7fffffff;
  for (int c = b; c < e; c++) {
    const int idx = Q.perm[c];
    if ((unsigned)idx >= (unsigned)Q.N) {  // uniform over the half warp
      if (l16 == 0) raise_status(Q.status, DEV_ERR_BOUNDS, g, c);
      continue;
    }
    const int x2 = idx % W, y2 = idx / W;
    const int cost = group_cost<R>(sc, Q.src.pitch, plane_centre(Q.tgt, x2, y2), Q.tgt.pitch, l16,
                                   gmask);
    if (cost < best || (cost == best && idx < bidx)) {
      best = cost;
      bidx = idx;
    }
  }
  // flows in units of 1/q pixel: leaf pixels and proposals (in pixels) scale by q
  const int lq = Q.tgt.log2q;
  uint32_t fbest = pack_flow((bidx % W - px) << lq, (bidx / W - py) << lq);
  for (int k = 0; k < Q.K; k++) {
    const uint32_t pr = Q.proposals[(size_t)g * Q.K + k];
    int X, Y;
    const uint32_t cf = clamp_target(Q.tgt, px, py, flow_dx(pr) << lq, flow_dy(pr) << lq, X, Y);
    const int cost = group_cost<R>(sc, Q.src.pitch, target_centre(Q.tgt, X, Y), Q.tgt.pitch, l16,
                                   gmask);
    if (cost < best) {
      best = cost;
      fbest = cf;
    }
  }
  if (l16 == 0) {
    Q.flow[g] = fbest;
    Q.cost[g] = best;
  }
}

ff_status launch_kd_query(const KdQuery *q, KdQuery *dev, int nq, cudaStream_t st) {
  if (nq <= 0) return FF_OK;
  FF_TRY(upload_desc(q, dev, nq, st));
  int r = q[0].r, maxG = 0;
  for (int i = 0; i < nq; i++) {
    if (q[i].r != r) return FF_ERR_INVALID_ARG;
    maxG = max(maxG, q[i].src.NX * q[i].src.NY);
  }
  dim3 grid((maxG * 16 + 255) / 256, nq);
  FF_DISPATCH_R(r, k_kd_query<RR><<<grid, 256, 0, st>>>(dev));
  FF_CHECK_LAUNCH();
  return FF_OK;
}

}  // namespace ff
