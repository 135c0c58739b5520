// C ABI of the library: argument checks, workspace planning and the per-pair
// orchestration of Fig. 2 (smoothed images and census for both frames, three
// flow fields each with its own kd tree, outlier filtering, sparsification).
//
// The three flows of a pair share every launch: kd builds, kd queries of equal
// radius, seeding and passes take an array of problems and index it with
// blockIdx.y, so one pair costs the same number of launches as one flow.
#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "ff_internal.cuh"

namespace ff {

// ------------------------------------------------------------ accounting -----
static std::atomic<uint64_t> g_launches{0};
static int g_prof = 0;  // bit 0: pass-kernel events, bit 1: evaluation counters, bit 2: phase marks
static std::vector<cudaEvent_t> g_ev;  // pairs (begin, end)
static std::vector<int> g_ev_tag;      // level (log2 n) of each pair
static size_t g_ev_used = 0;

// Candidate evaluations of the pass kernels, counted when profiling asks for it:
// [radius r][log2 n][kind], kinds as in PassCfg::evals. One array per device,
// filled by atomics at the end of every counted launch.
static __device__ unsigned long long g_evals[9 * PROF_LEVELS * 4];
static void *g_evals_ptr[64];
static std::mutex g_evals_mu;

static ff_status evals_ptr(unsigned long long **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FF_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_evals_mu);
  if (!g_evals_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_evals) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return FF_ERR_CUDA;
    }
    g_evals_ptr[dev] = p;
  }
  *out = (unsigned long long *)g_evals_ptr[dev];
  return FF_OK;
}

static ff_exec_params g_exec = {4, 0, 1, 2, 0, 0, 0, 0};
const ff_exec_params &exec_params() { return g_exec; }

void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
bool prof_enabled() { return (g_prof & 1) != 0; }
unsigned long long *prof_evals(int r, int log2n) {
  if (!(g_prof & 2) || r < 1 || r > 8 || log2n < 0 || log2n >= PROF_LEVELS) return nullptr;
  unsigned long long *p = nullptr;
  if (evals_ptr(&p) != FF_OK) return nullptr;
  return p + ((size_t)r * PROF_LEVELS + log2n) * 4;
}
void prof_begin(cudaStream_t s, int tag) {
  if (g_ev_used + 2 > g_ev.size()) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    g_ev.push_back(a);
    g_ev.push_back(b);
    g_ev_tag.push_back(0);
  }
  g_ev_tag[g_ev_used / 2] = tag;
  cudaEventRecord(g_ev[g_ev_used], s);
}
void prof_end(cudaStream_t s) {
  cudaEventRecord(g_ev[g_ev_used + 1], s);
  g_ev_used += 2;
}

// Phase marks of run_pairs: one timing event per phase boundary on the stream
// that ran the phase, tagged 100 * group + phase (group 3: the shared work).
static std::vector<cudaEvent_t> g_mark;
static std::vector<int> g_mark_tag;
static size_t g_mark_used = 0;
static void mark(cudaStream_t s, int group, int phase) {
  if (!(g_prof & 4)) return;
  if (g_mark_used == g_mark.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    g_mark.push_back(e);
    g_mark_tag.push_back(0);
  }
  g_mark_tag[g_mark_used] = 100 * group + phase;
  cudaEventRecord(g_mark[g_mark_used++], s);
}
enum { MK_START = 0, MK_PYRAMID = 1, MK_FEATURES = 2, MK_KD_BUILD = 3, MK_KD_QUERY = 4,
       MK_LEVEL = 10, MK_JOINED = 20, MK_FILTER = 21 };

// ------------------------------------------------------------ checks --------

ff_status check_params(const ff_params *p) {
  if (!p) return FF_ERR_INVALID_ARG;
  if (p->k < 0 || p->k > 4) return FF_ERR_INVALID_ARG;
  if (p->r < 1 || p->r > PLANE_PAD || p->r2 < 1 || p->r2 > PLANE_PAD) return FF_ERR_INVALID_ARG;
  if (p->leaf < 2 || p->leaf > 32) return FF_ERR_INVALID_ARG;
  if (p->R < 0 || p->R > 64) return FF_ERR_INVALID_ARG;
  if (p->eps < 1 || p->eps > 1000 || p->e < 1 || p->e > 9 || p->s < 0) return FF_ERR_INVALID_ARG;
  if (p->tile < 2 || p->tile > MAX_TILE || (p->tile & 1)) return FF_ERR_INVALID_ARG;
  if (p->n_rs < 0 || p->n_rs > 3 || p->K < 0 || p->K > MAX_K) return FF_ERR_INVALID_ARG;
  if (p->color < 0 || p->color > 1) return FF_ERR_INVALID_ARG;
  if (p->subpel != 1 && p->subpel != 2 && p->subpel != 4) return FF_ERR_INVALID_ARG;
  return FF_OK;
}

ff_status check_shape(int W, int H) {
  if (W < 1 || H < 1 || W > 16384 || H > 16384) return FF_ERR_SHAPE;
  if ((long long)W * H > (1ll << 24)) return FF_ERR_SHAPE;
  return FF_OK;
}

static std::mutex g_attr_mu;
static std::map<std::pair<int, const void *>, size_t> g_attr;

ff_status smem_opt_in(const void *func, size_t bytes) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return FF_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  size_t &have = g_attr[{dev, func}];
  if (bytes <= have) return FF_OK;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return FF_ERR_CUDA;
  }
  have = bytes;
  return FF_OK;
}




// ------------------------------------------------------------ pair plan ------
constexpr int MAXLV = 5;

struct PairPlan {
  uint8_t *lab[2];  // both frames in CIELab (params.color == 1), else null
  uint32_t *planes[2][MAXLV];
  uint8_t *sm[2];            // per frame: I^n, its smoothing scratch, its census
  void *smooth_scratch[2];
  uint32_t *census[2];
  int32_t *feat[3], *qfeat[3];
  int32_t *perm[3], *split_dim[3], *split_val[3];
  KdBuild kd[3];
  uint32_t *fa[3], *fb[3];
  int32_t *ca[3], *cb[3];
  void *filter_scratch;
};

// Per-pair scratch (everything but the workspace header and the descriptors).
static void plan_pair_body(Arena &a, int W, int H, const ff_params *p, PairPlan &P) {
  const size_t N = (size_t)W * H;
  for (int f = 0; f < 2; f++) P.lab[f] = p->color == 1 ? a.take<uint8_t>(N * 3) : nullptr;
  for (int f = 0; f < 2; f++)
    for (int lv = 0; lv <= p->k; lv++)
      P.planes[f][lv] = a.take<uint32_t>(planes_words(W, H, 1 << lv, p->subpel));
  size_t ss = 0;
  for (int lv = 1; lv <= p->k; lv++) ss = ss > smooth_scratch_bytes(W, H, 1 << lv) ? ss : smooth_scratch_bytes(W, H, 1 << lv);
  for (int f = 0; f < 2; f++) {
    P.sm[f] = a.take<uint8_t>(N * 3);
    P.smooth_scratch[f] = a.take<char>(ss);
    P.census[f] = a.take<uint32_t>(N);
  }
  const int ntop = 1 << p->k;
  const size_t Gtop = (size_t)((W + ntop - 1) / ntop) * ((H + ntop - 1) / ntop);
  const int D = kd_depth((int)N, p->leaf);
  for (int j = 0; j < 3; j++) {
    P.feat[j] = a.take<int32_t>(N * FEAT_PACKED_WORDS);  // packed rows (r <= 8)
    P.qfeat[j] = a.take<int32_t>(Gtop * FEAT_STRIDE);
    P.perm[j] = a.take<int32_t>(N);
    P.split_dim[j] = a.take<int32_t>((size_t)1 << D);
    P.split_val[j] = a.take<int32_t>((size_t)1 << D);
    KdBuild &b = P.kd[j];
    b = KdBuild{};
    b.N = (int)N;
    b.leaf = p->leaf;
    // WHT features of radius r: every dimension spans at most (2r+1)^2 * 255
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
    P.fa[j] = a.take<uint32_t>(N);
    P.fb[j] = a.take<uint32_t>(N);
    P.ca[j] = a.take<int32_t>(N);
    P.cb[j] = a.take<int32_t>(N);
  }
  P.filter_scratch = a.take<char>(filter_scratch_bytes(W, H));
}

// Workspace of a batch: header, every pair's scratch, then the descriptor
// arrays of the batched launches (3 flows per pair).
struct BatchDesc {
  KdBuild *d_kd;
  KdQuery *d_q;
  SearchProblem *d_sp;
  PyrJob *d_pyr;       // per level: the pyramid jobs (both frames of every pair)
  int32_t *tile_base;  // per level: tile prefix sums of the persistent level kernel
  unsigned *bar;       // per level: its grid-barrier counter (64 words apart)
};
static BatchDesc plan_batch(Arena &a, int np, const int *Ws, const int *Hs, const ff_params *p,
                            PairPlan *plans) {
  a.take<char>(WS_HEADER);
  for (int i = 0; i < np; i++) plan_pair_body(a, Ws[i], Hs[i], p, plans[i]);
  BatchDesc d;
  d.d_kd = a.take<KdBuild>(3 * (size_t)np);
  d.d_q = a.take<KdQuery>(3 * (size_t)np);
  d.d_sp = a.take<SearchProblem>(3 * (size_t)np * MAXLV);
  d.d_pyr = a.take<PyrJob>(2 * (size_t)np * MAXLV);
  d.tile_base = a.take<int32_t>((size_t)MAXLV * 2 * (3 * (size_t)np + 1));
  d.bar = a.take<unsigned>((size_t)MAXLV * 64);
  return d;
}

// One image pair's device buffers.
struct PairIO {
  const uint8_t *I1, *I2;
  int W, H;
  const int16_t *proposals;
  int16_t *flows;
  uint8_t *valid;
  int32_t *err_sum, *sparse, *n_sparse;
  uint8_t *mask;
};

// The whole path for np pairs (Fig. 2). Per-image kernels (smoothing, census,
// features, filtering) run per pair; the kd builds, kd queries and every search
// level of one flow (forward r, backward r, backward r2) take that flow's problems
// of all pairs in the same launches, each flow on a stream of its own.
static ff_status run_pairs(int np, const PairIO *io_in, const ff_params *p, void *ws,
                           size_t ws_bytes, cudaStream_t st) {
  std::vector<int> Ws(np), Hs(np);
  for (int i = 0; i < np; i++) {
    Ws[i] = io_in[i].W;
    Hs[i] = io_in[i].H;
  }
  std::vector<PairPlan> plans(np);
  Arena a(ws, ws_bytes);
  const BatchDesc bd = plan_batch(a, np, Ws.data(), Hs.data(), p, plans.data());
  if (!a.fits()) return FF_ERR_WORKSPACE;
  FF_TRY(clear_status(ws, st));
  // the colour space of every later step: the input channels, or both frames
  // converted to CIELab first
  std::vector<PairIO> io(io_in, io_in + np);
  if (p->color == 1)
    for (int i = 0; i < np; i++) {
      FF_TRY(launch_rgb_to_lab(io_in[i].I1, io[i].W, io[i].H, plans[i].lab[0], st));
      FF_TRY(launch_rgb_to_lab(io_in[i].I2, io[i].W, io[i].H, plans[i].lab[1], st));
      io[i].I1 = plans[i].lab[0];
      io[i].I2 = plans[i].lab[1];
    }
  const int k = p->k, ntop = 1 << k;
  const int srcf[3] = {0, 1, 1}, tgtf[3] = {1, 0, 0}, rad[3] = {p->r, p->r, p->r2};

  // problem order: the forward flows of every pair, then the first backward flows,
  // then the second backward flows. Each of these three groups computes its
  // features, builds its trees, queries them and searches on a stream of its own
  // (the caller's and two side streams), so the latency-bound kd builds and
  // searches of the three flows overlap.
  std::vector<int> order_pair, order_flow;
  for (int j = 0; j < 3; j++)
    for (int i = 0; i < np; i++) {
      order_pair.push_back(i);
      order_flow.push_back(j);
    }
  const int nprob = (int)order_pair.size();  // 3 * np
  const int ngroups = 3;
  // serial_flows (an execution parameter): every group on the caller's stream;
  // kd_merge: the kd trees of all groups are built in one launch chain on the
  // caller's stream before the groups fork
  const bool serial = exec_params().serial_flows != 0;
  const bool kd_merge = exec_params().kd_merge != 0;
  // persist_levels: one persistent launch per level over all problems (tiles of
  // edge <= 16, the CTA-per-tile pass form)
  const bool persist = exec_params().persist_levels != 0 && p->tile <= 16;
  SideSection sec;
  if (!serial) FF_TRY(sec.begin(st, 3));
  auto group_stream = [&](int g) { return (g == 0 || serial) ? st : sec.side[g - 1]; };
  // smoothed images and census planes of every pair (shared by all flows), on a
  // side stream of their own; the groups wait for them only before their kd
  // queries, so the pyramid overlaps their features and kd builds
  const cudaStream_t ps = serial ? st : sec.side[2];
  mark(st, 3, MK_START);
  // A batch runs one launch per step and level over both frames of every pair
  // (a 64-pair batch: 34 launches instead of 2,176, and the pyramid no longer
  // trails the kd builds). A single pair runs its frames one after the other, in
  // smaller launches that slot in beside the kd builds (measured faster there).
  std::vector<PyrJob> jobs(2 * (size_t)np);
  for (int lv = 0; lv <= k && np == 1; lv++) {
    const PairPlan &P = plans[0];
    const int W = io[0].W, H = io[0].H, n = 1 << lv;
    const uint8_t *img[2] = {io[0].I1, io[0].I2};
    for (int f = 0; f < 2; f++) {
      const uint8_t *src = img[f];
      if (n > 1) {
        FF_TRY(launch_smooth(img[f], W, H, n, P.sm[f], P.smooth_scratch[f], ps));
        src = P.sm[f];
      }
      const Planes pl = make_planes(P.planes[f][lv], W, H, n, p->subpel);
      FF_TRY(launch_census(src, W, H, n, P.census[f], ps));
      FF_TRY(launch_planes(P.census[f], phase_view(pl, 0), ps));
      for (int ph = 1; ph < p->subpel * p->subpel; ph++) {
        FF_TRY(launch_census_subpel(src, W, H, n, p->subpel, ph % p->subpel, ph / p->subpel,
                                    P.census[f], ps));
        FF_TRY(launch_planes(P.census[f], phase_view(pl, ph), ps));
      }
    }
  }
  for (int lv = 0; lv <= k && np > 1; lv++) {
    const int n = 1 << lv;
    for (int i = 0; i < np; i++) {
      const PairPlan &P = plans[i];
      const int W = io[i].W, H = io[i].H;
      const uint8_t *img[2] = {io[i].I1, io[i].I2};
      for (int f = 0; f < 2; f++) {
        const size_t Wc = (W + n - 1) / n, Hc = (H + n - 1) / n;
        PyrJob &J = jobs[2 * (size_t)i + f];
        J.img = img[f];
        J.down = (uint8_t *)P.smooth_scratch[f];
        J.h = (int32_t *)((char *)P.smooth_scratch[f] + ((Wc * Hc * 3 + 255) & ~(size_t)255));
        J.sm = P.sm[f];
        J.census = P.census[f];
        J.pl = phase_view(make_planes(P.planes[f][lv], W, H, n, p->subpel), 0);
        J.W = W;
        J.H = H;
      }
    }
    FF_TRY(launch_pyramid_level(jobs.data(), bd.d_pyr + 2 * (size_t)np * lv, 2 * np, n, ps));
    // subpixel targets (params.subpel > 1): the census of every other phase
    for (int i = 0; i < np && p->subpel > 1; i++) {
      const PairPlan &P = plans[i];
      const int W = io[i].W, H = io[i].H;
      for (int f = 0; f < 2; f++) {
        const uint8_t *src = n > 1 ? P.sm[f] : (f == 0 ? io[i].I1 : io[i].I2);
        const Planes pl = make_planes(P.planes[f][lv], W, H, n, p->subpel);
        for (int ph = 1; ph < p->subpel * p->subpel; ph++) {
          FF_TRY(launch_census_subpel(src, W, H, n, p->subpel, ph % p->subpel, ph / p->subpel,
                                      P.census[f], ps));
          FF_TRY(launch_planes(P.census[f], phase_view(pl, ph), ps));
        }
      }
    }
  }

  mark(ps, 3, MK_PYRAMID);
  if (!serial) FF_TRY(sec.signal(0, ps));

  std::vector<KdBuild> trees(nprob);
  std::vector<KdQuery> q(nprob);
  std::vector<uint32_t *> cur(nprob), oth(nprob);
  std::vector<int32_t *> ccur(nprob), coth(nprob);
  std::vector<SearchProblem> sp(nprob);
  for (int t = 0; t < nprob; t++) {
    const int i = order_pair[t], j = order_flow[t];
    const PairPlan &P = plans[i];
    const int W = io[i].W, H = io[i].H;
    trees[t] = P.kd[j];
    KdQuery &Q = q[t];
    Q = KdQuery{};
    Q.perm = P.perm[j];
    Q.split_dim = P.split_dim[j];
    Q.split_val = P.split_val[j];
    Q.N = W * H;
    Q.D = P.kd[j].D;
    Q.leaf = p->leaf;
    Q.qfeat = P.qfeat[j];
    Q.src = make_planes(P.planes[srcf[j]][k], W, H, ntop, p->subpel);
    Q.tgt = make_planes(P.planes[tgtf[j]][k], W, H, ntop, p->subpel);
    Q.r = rad[j];
    Q.proposals = (j == 0 && p->K > 0) ? (const uint32_t *)io[i].proposals : nullptr;
    Q.K = (j == 0) ? p->K : 0;
    Q.flow = P.fa[j];
    Q.cost = P.ca[j];
    Q.status = (DeviceStatus *)ws;
    cur[t] = P.fa[j];
    oth[t] = P.fb[j];
    ccur[t] = P.ca[j];
    coth[t] = P.cb[j];
  }
  // problem t's state at level lv: seeded from the coarser state (in cur) into the
  // other buffer below the coarsest level; the finest level writes the output flow
  auto level_problem = [&](int t, int lv) {
    const int i = order_pair[t], j = order_flow[t], n = 1 << lv;
    const PairPlan &P = plans[i];
    const int W = io[i].W, H = io[i].H;
    SearchProblem &s = sp[t];
    s = SearchProblem{};
    s.src = make_planes(P.planes[srcf[j]][lv], W, H, n, p->subpel);
    s.tgt = make_planes(P.planes[tgtf[j]][lv], W, H, n, p->subpel);
    s.r = rad[j];
    s.flow_id = j;
    if (lv == k) {
      s.flow_coarse = nullptr;
      s.flow_a = cur[t];
      s.cost_a = ccur[t];
      s.flow_b = oth[t];
      s.cost_b = coth[t];
    } else {
      s.flow_coarse = cur[t];
      s.flow_a = oth[t];
      s.cost_a = coth[t];
      s.flow_b = cur[t];
      s.cost_b = ccur[t];
    }
    if (lv == 0) {
      s.flow_final = (uint32_t *)(io[i].flows + 2 * (size_t)W * H * j);
      s.cost_final = s.cost_a;
    }
  };
  // WHT features of a group's target frames (all pixels) and source grid points
  auto group_features = [&](int g, cudaStream_t s) -> ff_status {
    for (int t = g * np; t < (g + 1) * np; t++) {
      const int i = order_pair[t], j = order_flow[t];
      const uint8_t *img[2] = {io[i].I1, io[i].I2};
      FF_TRY(launch_features(img[tgtf[j]], io[i].W, io[i].H, rad[j], nullptr, 0, 1,
                             plans[i].feat[j], s, true));
      FF_TRY(launch_features(img[srcf[j]], io[i].W, io[i].H, rad[j], nullptr, 0, ntop,
                             plans[i].qfeat[j], s));
    }
    return FF_OK;
  };
  if (kd_merge) {  // every tree in one launch chain, then the groups fork
    for (int g = 0; g < ngroups; g++) FF_TRY(group_features(g, st));
    mark(st, 3, MK_FEATURES);
    FF_TRY(launch_kd_build(trees.data(), bd.d_kd, nprob, st));
    mark(st, 3, MK_KD_BUILD);
    if (!serial) FF_TRY(sec.signal(1, st));
  }
  for (int g = 0; g < ngroups; g++) {
    const int t0 = g * np, cnt = np;
    cudaStream_t gs = group_stream(g);
    if (!kd_merge) {
      FF_TRY(group_features(g, gs));
      mark(gs, g, MK_FEATURES);
      FF_TRY(launch_kd_build(trees.data() + t0, bd.d_kd + t0, cnt, gs));
      mark(gs, g, MK_KD_BUILD);
    } else if (g != 0 && !serial) {
      FF_TRY(sec.wait(1, gs));  // trees built
    }
    if (!serial) FF_TRY(sec.wait(0, gs));  // census planes ready
    // kd query: one launch per run of equal radius
    for (int a0 = t0; a0 < t0 + cnt;) {
      int a1 = a0;
      while (a1 < t0 + cnt && q[a1].r == q[a0].r) a1++;
      FF_TRY(launch_kd_query(q.data() + a0, bd.d_q + a0, a1 - a0, gs));
      a0 = a1;
    }
    mark(gs, g, MK_KD_QUERY);
    if (persist) continue;  // the levels of all groups run below, one launch each
    // levels n = 2^k .. 1; the state alternates between the two buffers per level
    for (int lv = k; lv >= 0; lv--) {
      for (int t = t0; t < t0 + cnt; t++) level_problem(t, lv);
      FF_TRY(run_level_on(sp.data() + t0, bd.d_sp + (size_t)nprob * lv + t0, cnt, p->tile,
                          p->n_rs, p->R, p->seed, gs));
      mark(gs, g, MK_LEVEL + lv);
      if (lv != k)
        for (int t = t0; t < t0 + cnt; t++) {
          std::swap(cur[t], oth[t]);
          std::swap(ccur[t], coth[t]);
        }
    }
  }
  if (!serial) FF_TRY(sec.end());
  if (persist) {  // one persistent launch per level over every problem of the batch
    for (int lv = k; lv >= 0; lv--) {
      for (int t = 0; t < nprob; t++) level_problem(t, lv);
      FF_TRY(run_level_persistent(sp.data(), bd.d_sp + (size_t)nprob * lv, nprob,
                                  bd.tile_base + (size_t)lv * 2 * (nprob + 1), bd.bar + 64 * lv,
                                  (DeviceStatus *)ws, p->tile, p->n_rs, p->R, p->seed, st));
      mark(st, 3, MK_LEVEL + lv);
      if (lv != k)
        for (int t = 0; t < nprob; t++) {
          std::swap(cur[t], oth[t]);
          std::swap(ccur[t], coth[t]);
        }
    }
  }
  mark(st, 3, MK_JOINED);

  // the filters of a batch's pairs are independent: round-robin over the caller's
  // stream and the three side streams
  SideSection fsec;
  const bool fork = np > 1 && !serial;
  if (fork) FF_TRY(fsec.begin(st, 3));
  for (int i = 0; i < np; i++) {
    const size_t N = (size_t)io[i].W * io[i].H;
    const cudaStream_t fs = (!fork || i % 4 == 0) ? st : fsec.side[i % 4 - 1];
    FF_TRY(launch_filter((const uint32_t *)io[i].flows, (const uint32_t *)(io[i].flows + 2 * N),
                         (const uint32_t *)(io[i].flows + 4 * N), io[i].W, io[i].H, p->eps, p->e,
                         p->s, p->subpel, io[i].valid, io[i].err_sum, io[i].sparse, io[i].n_sparse,
                         io[i].mask, plans[i].filter_scratch, fs));
  }
  if (fork) FF_TRY(fsec.end());
  mark(st, 3, MK_FILTER);
  return FF_OK;
}

static size_t batch_ws_bytes(int np, const int *Ws, const int *Hs, const ff_params *p) {
  std::vector<PairPlan> plans(np);
  Arena a;
  plan_batch(a, np, Ws, Hs, p, plans.data());
  return a.off;
}

static ff_status check_pair(const PairIO &io, const ff_params *p) {
  FF_TRY(check_shape(io.W, io.H));
  // flows in units of 1/subpel pixel must fit int16
  if ((long long)(io.W - 1) * p->subpel > 32767 || (long long)(io.H - 1) * p->subpel > 32767)
    return FF_ERR_SHAPE;
  if (!io.I1 || !io.I2 || !io.flows || !io.valid || !io.err_sum || !io.sparse || !io.n_sparse ||
      !io.mask)
    return FF_ERR_INVALID_ARG;
  if (!aligned(io.flows, 4) || (p->K > 0 && !io.proposals) ||
      (io.proposals && !aligned(io.proposals, 4)))
    return FF_ERR_INVALID_ARG;
  return FF_OK;
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
  p->color = 0;
  p->subpel = 1;
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
  *bytes = batch_ws_bytes(1, &W, &H, p);
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
  q.status = (DeviceStatus *)ws;
  return launch_kd_query(&q, L.dq, 1, st);
}

ff_status ff_search_level(const uint32_t *census_src, const uint32_t *census_tgt, int W, int H,
                          int n, int r, const int16_t *flow_coarse, const ff_params *p,
                          int flow_id, int16_t *flow, int32_t *cost, void *ws, size_t ws_bytes,
                          void *stream) {
  FF_TRY(check_shape(W, H));
  FF_TRY(check_params(p));
  if (p->subpel != 1) return FF_ERR_INVALID_ARG;  // this entry takes one census per frame
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
                       p->eps, p->e, p->s, p->subpel, valid, err_sum, sparse, n_sparse, mask,
                       (char *)ws + WS_HEADER, st);
}

ff_status ff_flow_fields(const uint8_t *I1, const uint8_t *I2, int W, int H, const ff_params *p,
                         const int16_t *proposals, int16_t *flows, uint8_t *valid,
                         int32_t *err_sum, int32_t *sparse, int32_t *n_sparse, uint8_t *mask,
                         void *ws, size_t ws_bytes, void *stream) {
  FF_TRY(check_params(p));
  const PairIO io{I1, I2, W, H, proposals, flows, valid, err_sum, sparse, n_sparse, mask};
  FF_TRY(check_pair(io, p));
  FF_TRY(check_ws(ws, ws_bytes, batch_ws_bytes(1, &W, &H, p)));
  return run_pairs(1, &io, p, ws, ws_bytes, (cudaStream_t)stream);
}

static ff_status batch_io(int npairs, const ff_pair *pairs, const ff_params *p,
                          std::vector<PairIO> &io) {
  FF_TRY(check_params(p));
  if (npairs < 1 || npairs > FF_MAX_BATCH || !pairs) return FF_ERR_INVALID_ARG;
  io.resize(npairs);
  for (int i = 0; i < npairs; i++) {
    const ff_pair &q = pairs[i];
    io[i] = PairIO{q.I1, q.I2, q.W, q.H, q.proposals, q.flows, q.valid, q.err_sum, q.sparse,
                   q.n_sparse, q.mask};
    FF_TRY(check_pair(io[i], p));
  }
  return FF_OK;
}

ff_status ff_batch_workspace_size(int npairs, const ff_pair *pairs, const ff_params *p,
                                  size_t *bytes) {
  FF_TRY(check_params(p));
  if (npairs < 1 || npairs > FF_MAX_BATCH || !pairs || !bytes) return FF_ERR_INVALID_ARG;
  std::vector<int> Ws(npairs), Hs(npairs);
  for (int i = 0; i < npairs; i++) {
    FF_TRY(check_shape(pairs[i].W, pairs[i].H));
    Ws[i] = pairs[i].W;
    Hs[i] = pairs[i].H;
  }
  *bytes = batch_ws_bytes(npairs, Ws.data(), Hs.data(), p);
  return FF_OK;
}

ff_status ff_flow_fields_batch(int npairs, const ff_pair *pairs, const ff_params *p, void *ws,
                               size_t ws_bytes, void *stream) {
  std::vector<PairIO> io;
  FF_TRY(batch_io(npairs, pairs, p, io));
  size_t need;
  FF_TRY(ff_batch_workspace_size(npairs, pairs, p, &need));
  FF_TRY(check_ws(ws, ws_bytes, need));
  return run_pairs(npairs, io.data(), p, ws, ws_bytes, (cudaStream_t)stream);
}

struct ff_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  size_t kernels;
};

ff_status ff_graph_create(int npairs, const ff_pair *pairs, const ff_params *p, void *ws,
                          size_t ws_bytes, void *stream, ff_graph **out) {
  if (!out) return FF_ERR_INVALID_ARG;
  *out = nullptr;
  std::vector<PairIO> io;
  FF_TRY(batch_io(npairs, pairs, p, io));
  size_t need;
  FF_TRY(ff_batch_workspace_size(npairs, pairs, p, &need));
  FF_TRY(check_ws(ws, ws_bytes, need));
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return FF_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
  const int prof = g_prof;
  g_prof = 0;  // timing events cannot be read back from a graph
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    g_prof = prof;
    return FF_ERR_CUDA;
  }
  const ff_status rs = run_pairs(npairs, io.data(), p, ws, ws_bytes, st);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(st, &graph);
  g_prof = prof;
  if (rs != FF_OK || ce != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    (void)cudaGetLastError();
    return rs != FF_OK ? rs : FF_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return FF_ERR_CUDA;
  }
  size_t nn = 0;
  cudaGraphGetNodes(graph, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  size_t kern = 0;
  if (nn && cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
    for (size_t i = 0; i < nn; i++) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) kern++;
    }
  *out = new ff_graph{graph, exec, kern};
  return FF_OK;
}

ff_status ff_graph_launch(ff_graph *g, void *stream) {
  if (!g) return FF_ERR_INVALID_ARG;
  if (cudaGraphLaunch(g->exec, (cudaStream_t)stream) != cudaSuccess) return FF_ERR_CUDA;
  count_launch((int)g->kernels);
  return FF_OK;
}

ff_status ff_graph_kernel_count(const ff_graph *g, uint64_t *kernels) {
  if (!g || !kernels) return FF_ERR_INVALID_ARG;
  *kernels = g->kernels;
  return FF_OK;
}

ff_status ff_graph_destroy(ff_graph *g) {
  if (!g) return FF_OK;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
  return FF_OK;
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

ff_status ff_set_exec_params(const ff_exec_params *e) {
  auto pow2_or_0 = [](int v) { return v >= 0 && v <= 128 && (v & (v - 1)) == 0; };
  if (!e || e->pass_warps < 1 || e->pass_warps > 8 || !pow2_or_0(e->rs_min_n) ||
      !pow2_or_0(e->wide_min_n) || !pow2_or_0(e->split8_min_n) || e->serial_flows < 0 ||
      e->serial_flows > 1 || e->kd_merge < 0 || e->kd_merge > 1 || e->persist_levels < 0 ||
      e->persist_levels > 1 || !pow2_or_0(e->split2_max_n))
    return FF_ERR_INVALID_ARG;
  g_exec = *e;
  return FF_OK;
}

ff_status ff_set_wait_test(long long budget_cycles, int skip_block, int net_stall_polls) {
  if (budget_cycles < 0 || skip_block < -1 || net_stall_polls < 0) return FF_ERR_INVALID_ARG;
  set_wait_test(budget_cycles, skip_block, net_stall_polls);
  return FF_OK;
}

ff_status ff_get_exec_params(ff_exec_params *e) {
  if (!e) return FF_ERR_INVALID_ARG;
  *e = g_exec;
  return FF_OK;
}

ff_status ff_profile_enable(int on) {
  if (on < 0 || on > 7) return FF_ERR_INVALID_ARG;
  g_prof = on;
  return FF_OK;
}

ff_status ff_profile_reset(void) {
  g_launches.store(0);
  g_ev_used = 0;
  g_mark_used = 0;
  if (g_prof & 2) {
    unsigned long long *p = nullptr;
    FF_TRY(evals_ptr(&p));
    if (cudaMemset(p, 0, sizeof(g_evals)) != cudaSuccess) return FF_ERR_CUDA;
  }
  return FF_OK;
}

static ff_status event_ms(size_t i, double *ms) {
  if (cudaEventSynchronize(g_ev[i + 1]) != cudaSuccess) return FF_ERR_CUDA;
  float f = 0.f;
  if (cudaEventElapsedTime(&f, g_ev[i], g_ev[i + 1]) != cudaSuccess) return FF_ERR_CUDA;
  *ms = f;
  return FF_OK;
}

ff_status ff_profile_read(uint64_t *launches, double *prop_ms, uint64_t *prop_launches) {
  if (launches) *launches = g_launches.load();
  double tot = 0.0;
  for (size_t i = 0; i + 1 < g_ev_used; i += 2) {
    double ms;
    FF_TRY(event_ms(i, &ms));
    tot += ms;
  }
  if (prop_ms) *prop_ms = tot;
  if (prop_launches) *prop_launches = g_ev_used / 2;
  return FF_OK;
}

ff_status ff_profile_levels(double *ms, uint64_t *launches) {
  if (!ms || !launches) return FF_ERR_INVALID_ARG;
  for (int l = 0; l < PROF_LEVELS; l++) {
    ms[l] = 0.0;
    launches[l] = 0;
  }
  for (size_t i = 0; i + 1 < g_ev_used; i += 2) {
    const int l = g_ev_tag[i / 2];
    if (l < 0 || l >= PROF_LEVELS) continue;
    double t;
    FF_TRY(event_ms(i, &t));
    ms[l] += t;
    launches[l] += 1;
  }
  return FF_OK;
}

ff_status ff_profile_marks(int32_t *tags, double *ms, int cap, int *n) {
  if (!n || cap < 0 || (cap > 0 && (!tags || !ms))) return FF_ERR_INVALID_ARG;
  *n = (int)g_mark_used;
  if (g_mark_used == 0) return FF_OK;
  if (cudaEventSynchronize(g_mark[g_mark_used - 1]) != cudaSuccess) return FF_ERR_CUDA;
  for (size_t i = 0; i < g_mark_used && (int)i < cap; i++) {
    if (cudaEventSynchronize(g_mark[i]) != cudaSuccess) return FF_ERR_CUDA;
    float f = 0.f;
    if (cudaEventElapsedTime(&f, g_mark[0], g_mark[i]) != cudaSuccess) return FF_ERR_CUDA;
    tags[i] = g_mark_tag[i];
    ms[i] = f;
  }
  return FF_OK;
}

ff_status ff_profile_evals(uint64_t *counts) {
  if (!counts) return FF_ERR_INVALID_ARG;
  unsigned long long *p = nullptr;
  FF_TRY(evals_ptr(&p));
  if (cudaDeviceSynchronize() != cudaSuccess) return FF_ERR_CUDA;
  if (cudaMemcpy(counts, p, sizeof(g_evals), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FF_ERR_CUDA;
  return FF_OK;
}

}  // extern "C"
