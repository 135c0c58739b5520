// C ABI of the library: argument checks, workspace planning and the per-pair
// orchestration of Fig. 2 (smoothed images and census for both frames, three
// flow fields each with its own kd tree, outlier filtering, sparsification).
//
// The three flows of a pair share every launch: kd builds, kd queries of equal
// radius, seeding and passes take an array of problems and index it with
// blockIdx.y, so one pair costs the same number of launches as one flow.
#include <atomic>
#include <vector>

#include "ff_internal.cuh"

namespace ff {

// ------------------------------------------------------------ accounting -----
static std::atomic<uint64_t> g_launches{0};
static bool g_prof = false;
static std::vector<cudaEvent_t> g_ev;  // pairs (begin, end)
static size_t g_ev_used = 0;

void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
bool prof_enabled() { return g_prof; }
void prof_begin(cudaStream_t s) {
  if (g_ev_used + 2 > g_ev.size()) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    g_ev.push_back(a);
    g_ev.push_back(b);
  }
  cudaEventRecord(g_ev[g_ev_used], s);
}
void prof_end(cudaStream_t s) {
  cudaEventRecord(g_ev[g_ev_used + 1], s);
  g_ev_used += 2;
}

// ------------------------------------------------------------ checks --------
static bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

static ff_status check_params(const ff_params *p) {
  if (!p) return FF_ERR_INVALID_ARG;
  if (p->k < 0 || p->k > 4) return FF_ERR_INVALID_ARG;
  if (p->r < 1 || p->r > PLANE_PAD || p->r2 < 1 || p->r2 > PLANE_PAD) return FF_ERR_INVALID_ARG;
  if (p->leaf < 2 || p->leaf > 32) return FF_ERR_INVALID_ARG;
  if (p->R < 0 || p->R > 64) return FF_ERR_INVALID_ARG;
  if (p->eps < 1 || p->eps > 1000 || p->e < 1 || p->e > 9 || p->s < 0) return FF_ERR_INVALID_ARG;
  if (p->tile < 2 || p->tile > MAX_TILE || (p->tile & 1)) return FF_ERR_INVALID_ARG;
  if (p->n_rs < 0 || p->n_rs > 3 || p->K < 0 || p->K > MAX_K) return FF_ERR_INVALID_ARG;
  return FF_OK;
}

static ff_status check_shape(int W, int H) {
  if (W < 1 || H < 1 || W > 16384 || H > 16384) return FF_ERR_SHAPE;
  if ((long long)W * H > (1ll << 24)) return FF_ERR_SHAPE;
  return FF_OK;
}

static bool pow2_upto(int n, int hi) { return n >= 1 && n <= hi && (n & (n - 1)) == 0; }

static ff_status check_ws(void *ws, size_t have, size_t need) {
  if (need == 0) return FF_OK;
  if (!ws || !aligned(ws, 256)) return FF_ERR_WORKSPACE;
  if (have < need) return FF_ERR_WORKSPACE;
  return FF_OK;
}

static ff_status clear_status(void *ws, cudaStream_t st) {
  if (cudaMemsetAsync(ws, 0, sizeof(DeviceStatus), st) != cudaSuccess) return FF_ERR_CUDA;
  return FF_OK;
}

// ------------------------------------------------------------ pair plan ------
constexpr int MAXLV = 5;

struct PairPlan {
  uint32_t *planes[2][MAXLV];
  uint8_t *sm;
  void *smooth_scratch;
  uint32_t *census;
  int32_t *feat[3], *qfeat[3];
  int32_t *perm[3], *split_dim[3], *split_val[3];
  KdBuild kd[3];
  uint32_t *fa[3], *fb[3];
  int32_t *ca[3], *cb[3];
  void *filter_scratch;
  KdBuild *d_kd;
  KdQuery *d_q;
  SearchProblem *d_sp;
};

static void plan_pair(Arena &a, int W, int H, const ff_params *p, PairPlan &P) {
  const size_t N = (size_t)W * H;
  a.take<char>(WS_HEADER);
  for (int f = 0; f < 2; f++)
    for (int lv = 0; lv <= p->k; lv++) P.planes[f][lv] = a.take<uint32_t>(planes_words(W, H, 1 << lv));
  P.sm = a.take<uint8_t>(N * 3);
  size_t ss = 0;
  for (int lv = 1; lv <= p->k; lv++) ss = ss > smooth_scratch_bytes(W, H, 1 << lv) ? ss : smooth_scratch_bytes(W, H, 1 << lv);
  P.smooth_scratch = a.take<char>(ss);
  P.census = a.take<uint32_t>(N);
  const int ntop = 1 << p->k;
  const size_t Gtop = (size_t)((W + ntop - 1) / ntop) * ((H + ntop - 1) / ntop);
  const int D = kd_depth((int)N, p->leaf);
  for (int j = 0; j < 3; j++) {
    P.feat[j] = a.take<int32_t>(N * FEAT_STRIDE);
    P.qfeat[j] = a.take<int32_t>(Gtop * FEAT_STRIDE);
    P.perm[j] = a.take<int32_t>(N);
    P.split_dim[j] = a.take<int32_t>((size_t)1 << D);
    P.split_val[j] = a.take<int32_t>((size_t)1 << D);
    KdBuild &b = P.kd[j];
    b = KdBuild{};
    b.N = (int)N;
    b.leaf = p->leaf;
    kd_bind_scratch(b, a);
    b.feat = P.feat[j];
    b.perm = P.perm[j];
    b.split_dim = P.split_dim[j];
    b.split_val = P.split_val[j];
    b.status = (DeviceStatus *)a.base;
    P.fa[j] = a.take<uint32_t>(N);
    P.fb[j] = a.take<uint32_t>(N);
    P.ca[j] = a.take<int32_t>(N);
    P.cb[j] = a.take<int32_t>(N);
  }
  P.filter_scratch = a.take<char>(filter_scratch_bytes(W, H));
  P.d_kd = a.take<KdBuild>(3);
  P.d_q = a.take<KdQuery>(3);
  P.d_sp = a.take<SearchProblem>(3 * MAXLV);
}

}  // namespace ff

using namespace ff;

extern "C" {

const char *ff_status_str(ff_status s) {
  switch (s) {
    case FF_OK: return "ok";
    case FF_ERR_INVALID_ARG: return "invalid argument";
    case FF_ERR_SHAPE: return "unsupported image shape";
    case FF_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case FF_ERR_CUDA: return "CUDA error";
    case FF_ERR_DEVICE: return "device-side check failed";
  }
  return "unknown status";
}

ff_status ff_params_preset(ff_params *p, int preset) {
  if (!p) return FF_ERR_INVALID_ARG;
  *p = ff_params{};
  p->k = 3;
  p->r = 8;
  p->r2 = 6;
  p->leaf = 8;
  p->R = 1;
  p->tile = 16;
  p->n_rs = 3;
  p->K = 0;
  p->seed = 0;
  switch (preset) {
    case FF_PRESET_SINTEL: p->eps = 5; p->e = 4; p->s = 50; break;
    case FF_PRESET_MIDDLEBURY: p->eps = 1; p->e = 7; p->s = 50; break;
    case FF_PRESET_KITTI: p->eps = 1; p->e = 9; p->s = 150; break;
    default: return FF_ERR_INVALID_ARG;
  }
  return FF_OK;
}

ff_status ff_workspace_size(int W, int H, const ff_params *p, size_t *bytes) {
  FF_TRY(check_params(p));
  FF_TRY(check_shape(W, H));
  if (!bytes) return FF_ERR_INVALID_ARG;
  Arena a;
  PairPlan P;
  plan_pair(a, W, H, p, P);
  *bytes = a.off;
  return FF_OK;
}

ff_status ff_smooth_workspace_size(int W, int H, int n, size_t *bytes) {
  FF_TRY(check_shape(W, H));
  if (!bytes || !pow2_upto(n, 16)) return FF_ERR_INVALID_ARG;
  *bytes = smooth_scratch_bytes(W, H, n);
  return FF_OK;
}

ff_status ff_smooth(const uint8_t *img, int W, int H, int n, uint8_t *out, void *ws,
                    size_t ws_bytes, void *stream) {
  FF_TRY(check_shape(W, H));
  if (!img || !out || !pow2_upto(n, 16)) return FF_ERR_INVALID_ARG;
  FF_TRY(check_ws(ws, ws_bytes, smooth_scratch_bytes(W, H, n)));
  return launch_smooth(img, W, H, n, out, ws, (cudaStream_t)stream);
}

ff_status ff_census(const uint8_t *img_n, int W, int H, int n, uint32_t *out, void *stream) {
  FF_TRY(check_shape(W, H));
  if (!img_n || !out || !pow2_upto(n, 16) || !aligned(out, 4)) return FF_ERR_INVALID_ARG;
  return launch_census(img_n, W, H, n, out, (cudaStream_t)stream);
}

ff_status ff_features(const uint8_t *img, int W, int H, int r, const int32_t *pts, int npts,
                      int32_t *feat, void *stream) {
  FF_TRY(check_shape(W, H));
  if (!img || !feat || r < 1 || r > PLANE_PAD || !aligned(feat, 16)) return FF_ERR_INVALID_ARG;
  if (pts && npts < 0) return FF_ERR_INVALID_ARG;
  if (pts && npts == 0) return FF_OK;
  return launch_features(img, W, H, r, pts, npts, 1, feat, (cudaStream_t)stream);
}

ff_status ff_kdtree_size(int N, int leaf, int *depth, size_t *ws_bytes) {
  if (N < 1 || N > (1 << 24) || leaf < 2 || leaf > 32) return FF_ERR_INVALID_ARG;
  if (depth) *depth = kd_depth(N, leaf);
  if (ws_bytes) {
    Arena a;
    a.take<char>(WS_HEADER);
    a.take<KdBuild>(1);
    a.off += kd_scratch_bytes(N, leaf);
    *ws_bytes = a.off;
  }
  return FF_OK;
}

ff_status ff_kdtree_build(const int32_t *feat, int N, int leaf, int32_t *perm, int32_t *split_dim,
                          int32_t *split_val, void *ws, size_t ws_bytes, void *stream) {
  size_t need;
  FF_TRY(ff_kdtree_size(N, leaf, nullptr, &need));
  if (!feat || !perm || !split_dim || !split_val || !aligned(feat, 16)) return FF_ERR_INVALID_ARG;
  FF_TRY(check_ws(ws, ws_bytes, need));
  cudaStream_t st = (cudaStream_t)stream;
  Arena a(ws, ws_bytes);
  a.take<char>(WS_HEADER);
  KdBuild *dev = a.take<KdBuild>(1);
  KdBuild b{};
  b.N = N;
  b.leaf = leaf;
  kd_bind_scratch(b, a);
  b.feat = feat;
  b.perm = perm;
  b.split_dim = split_dim;
  b.split_val = split_val;
  b.status = (DeviceStatus *)ws;
  FF_TRY(clear_status(ws, st));
  return launch_kd_build(&b, dev, 1, st);
}

ff_status ff_level_workspace_size(int W, int H, int n, size_t *bytes) {
  FF_TRY(check_shape(W, H));
  if (!bytes || !pow2_upto(n, 16)) return FF_ERR_INVALID_ARG;
  const size_t G = (size_t)((W + n - 1) / n) * ((H + n - 1) / n);
  Arena a;
  a.take<char>(WS_HEADER);
  a.take<uint32_t>(planes_words(W, H, n));
  a.take<uint32_t>(planes_words(W, H, n));
  a.take<int32_t>(G * FEAT_STRIDE);
  a.take<uint32_t>(G);
  a.take<int32_t>(G);
  a.take<KdQuery>(1);
  a.take<SearchProblem>(1);
  *bytes = a.off;
  return FF_OK;
}

struct LevelWs {
  uint32_t *ps, *pt;
  int32_t *qfeat;
  uint32_t *fb;
  int32_t *cb;
  KdQuery *dq;
  SearchProblem *dsp;
};
static LevelWs bind_level_ws(void *ws, int W, int H, int n) {
  const size_t G = (size_t)((W + n - 1) / n) * ((H + n - 1) / n);
  Arena a(ws, (size_t)-1);
  a.take<char>(WS_HEADER);
  LevelWs L;
  L.ps = a.take<uint32_t>(planes_words(W, H, n));
  L.pt = a.take<uint32_t>(planes_words(W, H, n));
  L.qfeat = a.take<int32_t>(G * FEAT_STRIDE);
  L.fb = a.take<uint32_t>(G);
  L.cb = a.take<int32_t>(G);
  L.dq = a.take<KdQuery>(1);
  L.dsp = a.take<SearchProblem>(1);
  return L;
}

ff_status ff_kdtree_init(const int32_t *perm, const int32_t *split_dim, const int32_t *split_val,
                         int leaf, const uint8_t *src_img, const uint32_t *census_src,
                         const uint32_t *census_tgt, int W, int H, int n, int r,
                         const int16_t *proposals, int K, int16_t *flow, int32_t *cost, void *ws,
                         size_t ws_bytes, void *stream) {
  FF_TRY(check_shape(W, H));
  if (!perm || !split_dim || !split_val || !src_img || !census_src || !census_tgt || !flow || !cost)
    return FF_ERR_INVALID_ARG;
  if (leaf < 2 || leaf > 32 || !pow2_upto(n, 16) || r < 1 || r > PLANE_PAD) return FF_ERR_INVALID_ARG;
  if (K < 0 || K > MAX_K || (K > 0 && !proposals) || !aligned(flow, 4)) return FF_ERR_INVALID_ARG;
  size_t need;
  FF_TRY(ff_level_workspace_size(W, H, n, &need));
  FF_TRY(check_ws(ws, ws_bytes, need));
  cudaStream_t st = (cudaStream_t)stream;
  LevelWs L = bind_level_ws(ws, W, H, n);
  FF_TRY(clear_status(ws, st));
  Planes ps = make_planes(L.ps, W, H, n), pt = make_planes(L.pt, W, H, n);
  FF_TRY(launch_planes(census_src, ps, st));
  FF_TRY(launch_planes(census_tgt, pt, st));
  FF_TRY(launch_features(src_img, W, H, r, nullptr, 0, n, L.qfeat, st));
  KdQuery q{};
  q.perm = perm;
  q.split_dim = split_dim;
  q.split_val = split_val;
  q.N = W * H;
  q.D = kd_depth(W * H, leaf);
  q.leaf = leaf;
  q.qfeat = L.qfeat;
  q.src = ps;
  q.tgt = pt;
  q.r = r;
  q.proposals = (const uint32_t *)proposals;
  q.K = K;
  q.flow = (uint32_t *)flow;
  q.cost = cost;
  return launch_kd_query(&q, L.dq, 1, st);
}

ff_status ff_search_level(const uint32_t *census_src, const uint32_t *census_tgt, int W, int H,
                          int n, int r, const int16_t *flow_coarse, const ff_params *p,
                          int flow_id, int16_t *flow, int32_t *cost, void *ws, size_t ws_bytes,
                          void *stream) {
  FF_TRY(check_shape(W, H));
  FF_TRY(check_params(p));
  if (!census_src || !census_tgt || !flow || !cost || !aligned(flow, 4)) return FF_ERR_INVALID_ARG;
  if (flow_coarse && !aligned(flow_coarse, 4)) return FF_ERR_INVALID_ARG;
  if (!pow2_upto(n, 16) || r < 1 || r > PLANE_PAD || flow_id < 0 || flow_id > 3)
    return FF_ERR_INVALID_ARG;
  size_t need;
  FF_TRY(ff_level_workspace_size(W, H, n, &need));
  FF_TRY(check_ws(ws, ws_bytes, need));
  cudaStream_t st = (cudaStream_t)stream;
  LevelWs L = bind_level_ws(ws, W, H, n);
  FF_TRY(clear_status(ws, st));
  SearchProblem sp{};
  sp.src = make_planes(L.ps, W, H, n);
  sp.tgt = make_planes(L.pt, W, H, n);
  FF_TRY(launch_planes(census_src, sp.src, st));
  FF_TRY(launch_planes(census_tgt, sp.tgt, st));
  sp.r = r;
  sp.flow_id = flow_id;
  sp.flow_coarse = (const uint32_t *)flow_coarse;
  sp.flow_a = (uint32_t *)flow;
  sp.cost_a = cost;
  sp.flow_b = L.fb;
  sp.cost_b = L.cb;
  return run_level(&sp, L.dsp, 1, p->tile, p->n_rs, p->R, p->seed, st);
}

ff_status ff_filter_workspace_size(int W, int H, size_t *bytes) {
  FF_TRY(check_shape(W, H));
  if (!bytes) return FF_ERR_INVALID_ARG;
  *bytes = WS_HEADER + filter_scratch_bytes(W, H);
  return FF_OK;
}

ff_status ff_consistency_filter(const int16_t *F, const int16_t *Fb1, const int16_t *Fb2, int W,
                                int H, const ff_params *p, uint8_t *valid, int32_t *err_sum,
                                int32_t *sparse, int32_t *n_sparse, uint8_t *mask, void *ws,
                                size_t ws_bytes, void *stream) {
  FF_TRY(check_shape(W, H));
  FF_TRY(check_params(p));
  if (!F || !Fb1 || !Fb2 || !valid || !err_sum || !sparse || !n_sparse || !mask)
    return FF_ERR_INVALID_ARG;
  if (!aligned(F, 4) || !aligned(Fb1, 4) || !aligned(Fb2, 4)) return FF_ERR_INVALID_ARG;
  size_t need;
  FF_TRY(ff_filter_workspace_size(W, H, &need));
  FF_TRY(check_ws(ws, ws_bytes, need));
  cudaStream_t st = (cudaStream_t)stream;
  FF_TRY(clear_status(ws, st));
  return launch_filter((const uint32_t *)F, (const uint32_t *)Fb1, (const uint32_t *)Fb2, W, H,
                       p->eps, p->e, p->s, valid, err_sum, sparse, n_sparse, mask,
                       (char *)ws + WS_HEADER, st);
}

ff_status ff_flow_fields(const uint8_t *I1, const uint8_t *I2, int W, int H, const ff_params *p,
                         const int16_t *proposals, int16_t *flows, uint8_t *valid,
                         int32_t *err_sum, int32_t *sparse, int32_t *n_sparse, uint8_t *mask,
                         void *ws, size_t ws_bytes, void *stream) {
  FF_TRY(check_shape(W, H));
  FF_TRY(check_params(p));
  if (!I1 || !I2 || !flows || !valid || !err_sum || !sparse || !n_sparse || !mask)
    return FF_ERR_INVALID_ARG;
  if (!aligned(flows, 4) || (p->K > 0 && !proposals) || (proposals && !aligned(proposals, 4)))
    return FF_ERR_INVALID_ARG;
  size_t need;
  FF_TRY(ff_workspace_size(W, H, p, &need));
  FF_TRY(check_ws(ws, ws_bytes, need));
  cudaStream_t st = (cudaStream_t)stream;
  Arena a(ws, ws_bytes);
  PairPlan P;
  plan_pair(a, W, H, p, P);
  FF_TRY(clear_status(ws, st));
  const size_t N = (size_t)W * H;
  const int k = p->k, ntop = 1 << k;

  // smoothed images, census and phase planes of both frames at every level
  const uint8_t *img[2] = {I1, I2};
  for (int f = 0; f < 2; f++)
    for (int lv = 0; lv <= k; lv++) {
      const int n = 1 << lv;
      const uint8_t *src = img[f];
      if (n > 1) {
        FF_TRY(launch_smooth(img[f], W, H, n, P.sm, P.smooth_scratch, st));
        src = P.sm;
      }
      FF_TRY(launch_census(src, W, H, n, P.census, st));
      FF_TRY(launch_planes(P.census, make_planes(P.planes[f][lv], W, H, n), st));
    }

  // flow j: (source frame, target frame, radius): forward, backward r, backward r2
  const int srcf[3] = {0, 1, 1}, tgtf[3] = {1, 0, 0}, rad[3] = {p->r, p->r, p->r2};
  for (int j = 0; j < 3; j++) {
    FF_TRY(launch_features(img[tgtf[j]], W, H, rad[j], nullptr, 0, 1, P.feat[j], st));
    FF_TRY(launch_features(img[srcf[j]], W, H, rad[j], nullptr, 0, ntop, P.qfeat[j], st));
  }
  FF_TRY(launch_kd_build(P.kd, P.d_kd, 3, st));

  KdQuery q[3];
  for (int j = 0; j < 3; j++) {
    q[j] = KdQuery{};
    q[j].perm = P.perm[j];
    q[j].split_dim = P.split_dim[j];
    q[j].split_val = P.split_val[j];
    q[j].N = (int)N;
    q[j].D = P.kd[j].D;
    q[j].leaf = p->leaf;
    q[j].qfeat = P.qfeat[j];
    q[j].src = make_planes(P.planes[srcf[j]][k], W, H, ntop);
    q[j].tgt = make_planes(P.planes[tgtf[j]][k], W, H, ntop);
    q[j].r = rad[j];
    q[j].proposals = (j == 0 && p->K > 0) ? (const uint32_t *)proposals : nullptr;
    q[j].K = (j == 0) ? p->K : 0;
    q[j].flow = P.fa[j];
    q[j].cost = P.ca[j];
  }
  if (p->r == p->r2) {
    FF_TRY(launch_kd_query(q, P.d_q, 3, st));
  } else {
    FF_TRY(launch_kd_query(q, P.d_q, 2, st));
    FF_TRY(launch_kd_query(q + 2, P.d_q + 2, 1, st));
  }

  // levels n = 2^k .. 1; the state alternates between the two buffers per level
  uint32_t *cur[3], *oth[3];
  int32_t *ccur[3], *coth[3];
  for (int j = 0; j < 3; j++) {
    cur[j] = P.fa[j];
    oth[j] = P.fb[j];
    ccur[j] = P.ca[j];
    coth[j] = P.cb[j];
  }
  for (int lv = k; lv >= 0; lv--) {
    const int n = 1 << lv;
    SearchProblem sp[3];
    for (int j = 0; j < 3; j++) {
      SearchProblem &s = sp[j];
      s = SearchProblem{};
      s.src = make_planes(P.planes[srcf[j]][lv], W, H, n);
      s.tgt = make_planes(P.planes[tgtf[j]][lv], W, H, n);
      s.r = rad[j];
      s.flow_id = j;
      if (lv == k) {
        s.flow_coarse = nullptr;
        s.flow_a = cur[j];
        s.cost_a = ccur[j];
        s.flow_b = oth[j];
        s.cost_b = coth[j];
      } else {  // seed from the coarser state (in cur) into the other buffer
        s.flow_coarse = cur[j];
        s.flow_a = oth[j];
        s.cost_a = coth[j];
        s.flow_b = cur[j];
        s.cost_b = ccur[j];
      }
      if (lv == 0) {
        s.flow_final = (uint32_t *)(flows + 2 * N * j);
        s.cost_final = s.cost_a;
      }
    }
    FF_TRY(run_level(sp, P.d_sp + 3 * lv, 3, p->tile, p->n_rs, p->R, p->seed, st));
    if (lv != k)
      for (int j = 0; j < 3; j++) {
        uint32_t *t = cur[j];
        cur[j] = oth[j];
        oth[j] = t;
        int32_t *c = ccur[j];
        ccur[j] = coth[j];
        coth[j] = c;
      }
  }

  return launch_filter((const uint32_t *)flows, (const uint32_t *)(flows + 2 * N),
                       (const uint32_t *)(flows + 4 * N), W, H, p->eps, p->e, p->s, valid,
                       err_sum, sparse, n_sparse, mask, P.filter_scratch, st);
}

ff_status ff_device_status(const void *ws, uint32_t *code, int32_t *x, int32_t *y, void *stream) {
  if (!ws) return FF_ERR_INVALID_ARG;
  DeviceStatus h{};
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FF_ERR_CUDA;
  if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return FF_ERR_CUDA;
  if (code) *code = h.code;
  if (x) *x = h.x;
  if (y) *y = h.y;
  return h.code == DEV_OK ? FF_OK : FF_ERR_DEVICE;
}

ff_status ff_profile_enable(int on) {
  g_prof = on != 0;
  return FF_OK;
}

ff_status ff_profile_reset(void) {
  g_launches.store(0);
  g_ev_used = 0;
  return FF_OK;
}

ff_status ff_profile_read(uint64_t *launches, double *prop_ms, uint64_t *prop_launches) {
  if (launches) *launches = g_launches.load();
  double tot = 0.0;
  for (size_t i = 0; i + 1 < g_ev_used; i += 2) {
    if (cudaEventSynchronize(g_ev[i + 1]) != cudaSuccess) return FF_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g_ev[i], g_ev[i + 1]) != cudaSuccess) return FF_ERR_CUDA;
    tot += ms;
  }
  if (prop_ms) *prop_ms = tot;
  if (prop_launches) *prop_launches = g_ev_used / 2;
  return FF_OK;
}

}  // extern "C"
