// Sec. 3.1 / 3.2: hierarchical propagation (Eq. 2) and random search at one level.
//
// Seeding (level transition): a grid point with both coordinates even takes the
// flow of the coarser level with E_d re-evaluated here; every other point starts
// without a flow (cost 0x7fffffff).
//
// Pass kernel: one warp per T x T tile of grid points, pass_warps tiles per CTA
// (an execution parameter). The fixed parallel schedule: inside the tile the pass
// is exactly the sequential scan of the pass's direction, and a source outside
// the tile is read from the state at the start of the pass; odd passes shift the
// tile origin by T/2. Since a point depends only on its two source neighbours,
// the scan is run as anti-diagonal wavefronts: lane j owns scan row j (for
// T <= 16 lane j + 16 evaluates that row's vertical candidate concurrently), and
// one diagonal step per lane evaluates the candidates of its point and applies
// them in the order current, horizontal, vertical with strict-less replacement.
// A propagation candidate whose target is not clamped is costed incrementally:
// the patch of p under q's flow differs from q's by one line, so
// E(p, f) = E(q, f) - outgoing line + incoming line, exactly. After the wavefront
// the random search of the pass (if any) runs on all tile points, one lane per
// point, with offsets from the counter-based generator.
// Per tile and pass, shared memory holds: the source window (the tile's patches
// in the source frame's phase-(0,0) plane), a target window around where the
// tile centre's flow lands (hit by most candidates of a coherent field), the tile
// state and the state of the neighbours just outside the tile. Targets outside
// the window are gathered from the census phase planes (column lines from the
// transposed planes), through L1/L2.
#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "ff_internal.cuh"

namespace ff {

// Sources of each pass: (dx, dy) of the horizontal, then vertical neighbour.
__constant__ int c_pass_src[4][2][2] = {
    {{-1, 0}, {0, -1}}, {{1, 0}, {0, 1}}, {{1, 0}, {0, -1}}, {{-1, 0}, {0, 1}}};

// Level seeding. One 16-lane group per 2x2 block of grid points (grid-stride):
// the even-even point takes the coarse flow and its E_d at this level, the other
// three start unset. seed_block handles block c (coarse grid point c) of P.
template <int R>
__device__ __forceinline__ void seed_block(const SearchProblem &P, int c, int l16, unsigned gmask) {
  const int NX = P.src.NX, NY = P.src.NY, n = P.src.n;
  const int NXc = (NX + 1) >> 1;
  const int gx = (c % NXc) * 2, gy = (c / NXc) * 2;
  if (l16 >= 1 && l16 <= 3) {
    const int ox = gx + (l16 & 1), oy = gy + (l16 >> 1);
    if (ox < NX && oy < NY) {
      P.flow_a[(size_t)oy * NX + ox] = 0;
      P.cost_a[(size_t)oy * NX + ox] = COST_UNSET;
    }
  }
  const uint32_t f = P.flow_coarse[c];
  const int px = gx * n, py = gy * n;
  int X, Y;
  const uint32_t cf = clamp_target(P.tgt, px, py, f, X, Y);
  const int cost = group_cost<R>(plane_centre(P.src, px, py), P.src.pitch,
                                 target_centre(P.tgt, X, Y), P.tgt.pitch, l16, gmask);
  if (l16 == 0) {
    P.flow_a[(size_t)gy * NX + gx] = cf;
    P.cost_a[(size_t)gy * NX + gx] = cost;
  }
}
// Coarse grid points (= 2x2 blocks of this level) of a seeded problem.
__device__ __forceinline__ int seed_blocks(const SearchProblem &P) {
  return ((P.src.NX + 1) >> 1) * ((P.src.NY + 1) >> 1);
}

template <int R>
__global__ void __launch_bounds__(256) k_seed(const SearchProblem *probs) {
  const SearchProblem &P = probs[blockIdx.y];
  const int Gc = seed_blocks(P);
  const int l16 = threadIdx.x & 15;
  const unsigned gmask = 0xffffu << (threadIdx.x & 16);
  const int stride = (gridDim.x * blockDim.x) >> 4;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 4; c < Gc; c += stride)
    seed_block<R>(P, c, l16, gmask);
}

// Random search of pass s as a kernel of its own (levels where the execution
// parameters ask for it): one 16-lane group per grid point, in place on the
// pass's output. A point's random search reads and writes only its own state, so
// this equals the in-pass form exactly.
template <int R>
__global__ void __launch_bounds__(256) k_rs(const SearchProblem *probs, int s, int Rfull,
                                            uint64_t seed, unsigned long long *evals) {
  const SearchProblem &P = probs[blockIdx.y];
  const int NX = P.src.NX, G = NX * P.src.NY, n = P.src.n, log2n = P.src.log2n;
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int l16 = threadIdx.x & 15;
  const unsigned gmask = 0xffffu << (threadIdx.x & 16);
  if (g >= G) return;
  uint32_t *fl = (s & 1) ? P.flow_a : P.flow_b;  // the pass's output buffers
  int32_t *co = (s & 1) ? P.cost_a : P.cost_b;
  const int32_t cc = co[g];
  if (cc == COST_UNSET) return;
  const uint32_t cur = fl[g];
  const int gx = g % NX, gy = g / NX, px = gx * n, py = gy * n;
  int ox, oy, X, Y;
  rs_offset(seed, P.flow_id, log2n, s, gx, gy, (Rfull * n) << P.tgt.log2q, ox, oy);
  const uint32_t cf = clamp_target(P.tgt, px, py, flow_dx(cur) + ox, flow_dy(cur) + oy, X, Y);
  if (cf == cur) return;
  const int cost = group_cost<R>(plane_centre(P.src, px, py), P.src.pitch,
                                 target_centre(P.tgt, X, Y), P.tgt.pitch, l16, gmask);
  if (l16 == 0 && cost < cc) {
    fl[g] = cf;
    co[g] = cost;
  }
  if (evals && l16 == 0) atomicAdd(evals + 3, 1ull);
}

struct PassCfg {
  int s;        // pass 0..3
  int tile;     // T
  int do_rs;    // random search after this pass
  int R;        // full-resolution random-search radius
  uint64_t seed;
  int last;     // last pass of the level (writes flow_final when given)
  int words_per_tile;  // shared memory words of one tile
  // nullptr, or counters this launch adds its candidate evaluations to, by kind:
  // [0] incremental with the target in the staged window, [1] incremental with
  // the target read from the planes, [2] full E_d in the window, [3] full E_d
  // from the planes (an incremental evaluation reads 2 (2r+1) target taps, a full
  // one (2r+1)^2)
  unsigned long long *evals;
};

// Evaluation counting (profiling only): a launch with cfg.evals set adds every
// evaluation to four shared-memory counters (kinds as above) placed after the
// tiles, and flushes them to cfg.evals at its end; without it the kernels only
// test the uniform pointer.
__device__ __forceinline__ void count_eval(unsigned *scnt, bool full, bool window) {
  atomicAdd(scnt + (full ? 2 : 0) + (window ? 0 : 1), 1u);
}

constexpr int PASS_MAX_WARPS = 8;  // tiles per CTA: an execution parameter, 1..8
constexpr unsigned FULL_MASK = 0xffffffffu;

// Shared-memory layout of one tile (all sizes in 32-bit words). Both windows use
// odd pitches. (Pitches of 2 mod 4 with the random search's points taken column
// by column halve the shared-memory bank conflicts of the 16 x 16 tile, but
// measured slower: 4.24 against 4.20 ms per 1024x436 pair.)
struct TileLayout {
  int sw, swp;   // source window edge and pitch
  int tw, twp;   // target window edge and pitch
  int T;
  __host__ __device__ TileLayout(int T_, int R) : T(T_) {
    sw = T_ + 2 * R + 2;
    tw = T_ + 2 * R + 8;  // 3 entries of slack on each side of the tile's patches
    swp = sw | 1;
    twp = tw | 1;
  }
  __host__ __device__ int words() const { return sw * swp + tw * twp + 2 * T * T + 4 * T; }
};

// Shared-memory regions of one tile (all sizes in 32-bit words): source window,
// target window, tile state, and the state of the neighbours just outside the
// tile (horizontal: one per row, vertical: one per column).
struct TileSmem {
  uint32_t *src, *tgt, *flow;
  int32_t *cost;
  uint32_t *hf;
  int32_t *hc;
  uint32_t *vf;
  int32_t *vc;
};

__device__ __forceinline__ TileSmem carve_tile(uint32_t *base, const TileLayout &Lt, int T) {
  TileSmem S;
  S.src = base;
  S.tgt = S.src + Lt.sw * Lt.swp;
  S.flow = S.tgt + Lt.tw * Lt.twp;
  S.cost = (int32_t *)(S.flow + T * T);
  S.hf = (uint32_t *)(S.cost + T * T);
  S.hc = (int32_t *)(S.hf + T);
  S.vf = (uint32_t *)(S.hc + T);
  S.vc = (int32_t *)(S.vf + T);
  return S;
}

// Copies a tile's state, its outside neighbours, its source window and its
// target window into shared memory; threads sl, sl + width, ... share the work.
// The target window is where the tile's patches land under the flow of a set
// point near the tile centre (after seeding the even-even points are set); it
// is one phase plane's window, ph0 < 0 when there is none.
template <int R>
__device__ __forceinline__ void stage_tile(const SearchProblem &P, const TileLayout &Lt, int T,
                                           bool live, int x0, int y0, int x1, int y1, int hdx,
                                           int vdy, const uint32_t *fin, const int32_t *cin,
                                           const TileSmem &S, int sl, int width, int &tox,
                                           int &toy, int &ph0) {
  const int Gx = P.src.NX, Gy = P.src.NY, n = P.src.n;
  const int tw = live ? x1 - x0 : 0, th = live ? y1 - y0 : 0;
  for (int i = sl; i < tw * th; i += width) {
    const int lx = i % tw, ly = i / tw;
    const size_t g = (size_t)(y0 + ly) * Gx + x0 + lx;
    S.flow[ly * T + lx] = fin[g];
    S.cost[ly * T + lx] = cin[g];
  }
  if (live) {
    const int hx = hdx < 0 ? x0 - 1 : x1, vy = vdy < 0 ? y0 - 1 : y1;
    for (int i = sl; i < th; i += width) {
      const bool ok = hx >= 0 && hx < Gx;
      S.hf[i] = ok ? fin[(size_t)(y0 + i) * Gx + hx] : 0u;
      S.hc[i] = ok ? cin[(size_t)(y0 + i) * Gx + hx] : COST_UNSET;
    }
    for (int i = sl; i < tw; i += width) {
      const bool ok = vy >= 0 && vy < Gy;
      S.vf[i] = ok ? fin[(size_t)vy * Gx + x0 + i] : 0u;
      S.vc[i] = ok ? cin[(size_t)vy * Gx + x0 + i] : COST_UNSET;
    }
  }
  {
    const int ww = live ? tw + 2 * R + 2 : 0, wh = th + 2 * R + 2;
    const int ex0 = x0 - R - 1 + PLANE_PAD, ey0 = y0 - R - 1 + PLANE_PAD;
    for (int i = sl; i < ww * wh; i += width) {
      const int wx = i % ww, wy = i / ww;
      const int ex = ex0 + wx, ey = ey0 + wy;
      // entries outside the plane are only reachable through neighbours outside
      // the grid, which are never used
      S.src[wy * Lt.swp + wx] = (ex >= 0 && ey >= 0 && ex < P.src.pitch && ey < P.src.rows)
                                    ? P.src.base[(size_t)ey * P.src.pitch + ex]
                                    : 0u;
    }
  }
  tox = 0;
  toy = 0;
  ph0 = -1;
  if (live) {
    int gx = x0 + (tw >> 1), gy = y0 + (th >> 1);
    if (cin[(size_t)gy * Gx + gx] == COST_UNSET) {
      gx &= ~1;
      gy &= ~1;
    }
    const size_t g = (size_t)gy * Gx + gx;
    if (cin[g] != COST_UNSET) {
      const uint32_t fc = fin[g];
      const int X = ((gx * n) << P.tgt.log2q) + flow_dx(fc), Y = ((gy * n) << P.tgt.log2q) + flow_dy(fc);
      int cex, cey;
      target_plane(P.tgt, X, Y, ph0, cex, cey);  // shifts floor: X, Y may be outside
      const int slack = Lt.tw - (tw + 2 * R + 2);
      tox = (x0 - R - 1) + (cex - gx) - slack / 2;
      toy = (y0 - R - 1) + (cey - gy) - slack / 2;
    }
  }
  if (ph0 >= 0) {
    const uint32_t *pl = P.tgt.base + (size_t)ph0 * P.tgt.plane_words;
    const int tpitch = P.tgt.pitch, trows = P.tgt.rows;
    for (int i = sl; i < Lt.tw * Lt.tw; i += width) {
      const int wx = i % Lt.tw, wy = i / Lt.tw;
      const int ex = tox + wx, ey = toy + wy;
      // entries outside the plane are never inside a valid candidate's patch
      S.tgt[wy * Lt.twp + wx] = (ex >= 0 && ey >= 0 && ex < tpitch && ey < trows)
                                    ? pl[(size_t)ey * tpitch + ex]
                                    : 0u;
    }
  }
}

// Incremental E_d delta of a propagation candidate, by one lane. When p takes the
// flow f of its neighbour q = p + s*n along one axis and the target is not
// clamped, the patches of p and q (and of p + f, q + f) differ by one line:
//   E(p, f) = E(q, f) - E_line(q side) + E_line(p side)   (exact in integers).
// so_/si_ and to_/ti_ point at the first tap of the outgoing/incoming line in the
// source window and in the target (window or plane); ss/ts are the strides along
// the line. Horizontal neighbours give column lines, vertical ones row lines;
// both use this one loop, so lanes of a warp never split on the direction.
template <int R>
__device__ __forceinline__ int lane_line_delta(const uint32_t *so_, const uint32_t *si_, int ss,
                                               const uint32_t *to_, const uint32_t *ti_, int ts) {
  // two independent accumulators per line keep the add chains short
  int in0 = 0, in1 = 0, out0 = 0, out1 = 0;
#pragma unroll
  for (int w = 0; w < 2 * R + 1; w++) {
    const int pi = __popc(si_[w * ss] ^ ti_[w * ts]), po = __popc(so_[w * ss] ^ to_[w * ts]);
    if (w & 1) {
      in1 += pi;
      out1 += po;
    } else {
      in0 += pi;
      out0 += po;
    }
  }
  return (in0 + in1) - (out0 + out1);
}

// Full E_d by one lane; rows of the source window and of the target. Four
// accumulators break the chain of dependent adds across the (2R+1)^2 taps.
template <int R>
__device__ __forceinline__ int lane_full(const uint32_t *sc, int swp, const uint32_t *tc, int tp) {
  int a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  sc -= R * swp + R;
  tc -= R * tp + R;
#pragma unroll 3
  for (int v = 0; v < 2 * R + 1; v++) {
#pragma unroll
    for (int u = 0; u < 2 * R + 1; u++) {
      const int pc = __popc(sc[u] ^ tc[u]);
      switch (u & 3) {
        case 0: a0 += pc; break;
        case 1: a1 += pc; break;
        case 2: a2 += pc; break;
        default: a3 += pc; break;
      }
    }
    sc += swp;
    tc += tp;
  }
  return (a0 + a1) + (a2 + a3);
}

template <int R>
__global__ void __launch_bounds__(PASS_MAX_WARPS * 32) k_pass(const SearchProblem *probs, PassCfg cfg) {
  extern __shared__ uint32_t smem[];
  const SearchProblem &P = probs[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tpw = 1, width = 32, sub = 0, sl = lane;
  const int Gx = P.src.NX, Gy = P.src.NY, n = P.src.n, log2n = P.src.log2n;
  const int T = cfg.tile, off = (cfg.s & 1) * (T >> 1);
  const int ntx = (Gx + off + T - 1) / T, nty = (Gy + off + T - 1) / T;
  const int tile = (blockIdx.x * (blockDim.x >> 5) + warp) * tpw + sub;
  const bool live = tile < ntx * nty;
  if (!__any_sync(FULL_MASK, live)) return;  // whole warp; no block barriers below
  const int tx = live ? tile % ntx : 0, ty = live ? tile / ntx : 0;
  const int x0 = max(tx * T - off, 0), x1 = min(tx * T - off + T, Gx);
  const int y0 = max(ty * T - off, 0), y1 = min(ty * T - off + T, Gy);
  const int tw = live ? x1 - x0 : 0, th = live ? y1 - y0 : 0;
  const int hdx = c_pass_src[cfg.s][0][0], vdy = c_pass_src[cfg.s][1][1];
  const TileLayout Lt(T, R);

  const uint32_t *fin = (cfg.s & 1) ? P.flow_b : P.flow_a;
  const int32_t *cin = (cfg.s & 1) ? P.cost_b : P.cost_a;
  uint32_t *fout = (cfg.s & 1) ? P.flow_a : P.flow_b;
  int32_t *cout = (cfg.s & 1) ? P.cost_a : P.cost_b;
  if (cfg.last && P.flow_final) {
    fout = P.flow_final;
    cout = P.cost_final;
  }
  const uint32_t *tbase = P.tgt.base, *tbaseT = P.tgt.baseT;
  const int tpitch = P.tgt.pitch, tpitchT = P.tgt.pitchT;
  const size_t tpw_ = P.tgt.plane_words, tpwT = P.tgt.plane_wordsT;

  const TileSmem S = carve_tile(smem + (size_t)(warp * tpw + sub) * cfg.words_per_tile, Lt, T);
  uint32_t *s_src = S.src, *s_tgt = S.tgt, *s_flow = S.flow;
  int32_t *s_cost = S.cost;
  const uint32_t *s_hf = S.hf, *s_vf = S.vf;
  const int32_t *s_hc = S.hc, *s_vc = S.vc;
  int tox = 0, toy = 0, ph0 = -1;
  stage_tile<R>(P, Lt, T, live, x0, y0, x1, y1, hdx, vdy, fin, cin, S, sl, width, tox, toy, ph0);
  __syncwarp();

  // target of candidate flow f at pixel (px, py): plane phase and entry; in_win
  // when the whole patch plus one line lies inside this tile's target window
  struct Tgt {
    int ph, ex, ey;
    bool win;
  };
  auto locate = [&](int px, int py, uint32_t f) {  // f: a clamped flow
    Tgt t;
    target_plane(P.tgt, (px << P.tgt.log2q) + flow_dx(f), (py << P.tgt.log2q) + flow_dy(f), t.ph,
                 t.ex, t.ey);
    t.win = t.ph == ph0 && t.ex - R - 1 >= tox && t.ex + R + 1 < tox + Lt.tw &&
            t.ey - R - 1 >= toy && t.ey + R + 1 < toy + Lt.tw;
    return t;
  };

  // Propagation candidate c (0: horizontal source, 1: vertical source) of the
  // point at scan position (ip, jp): its clamped flow, whether it is worth
  // evaluating, and its E_d (incremental when the flow is unchanged by clamping).
  // evaluation counters (PassCfg::evals): four words per warp after the CTA's tiles
  unsigned *scnt = smem + (size_t)(blockDim.x >> 5) * tpw * cfg.words_per_tile + 4 * warp;
  if (cfg.evals && lane < 4) scnt[lane] = 0;
  auto evaluate = [&](int c, int lx, int ly, int px, int py, uint32_t fq, int32_t cq, int &cost) {
    const uint32_t *sc = s_src + (ly + R + 1) * Lt.swp + (lx + R + 1);
    int X, Y;
    const uint32_t cf = clamp_target(P.tgt, px, py, fq, X, Y);
    const Tgt t = locate(px, py, cf);
    if (cfg.evals) count_eval(scnt, cf != fq, t.win);
    if (cf == fq) {
      const int step = c == 0 ? hdx : vdy;
      const int oo = step + step * R, oi = -step * R;  // outgoing / incoming line offsets
      const uint32_t *so_, *si_, *to_, *ti_;
      int ss, ts;
      if (c == 0) {  // column lines
        ss = Lt.swp;
        so_ = sc - R * Lt.swp + oo;
        si_ = sc - R * Lt.swp + oi;
        if (t.win) {
          const uint32_t *tc = s_tgt + (t.ey - toy) * Lt.twp + (t.ex - tox);
          ts = Lt.twp;
          to_ = tc - R * Lt.twp + oo;
          ti_ = tc - R * Lt.twp + oi;
        } else {  // rows of the transposed plane
          const uint32_t *tc = tbaseT + (size_t)t.ph * tpwT + (size_t)t.ex * tpitchT + t.ey;
          ts = 1;
          to_ = tc + oo * tpitchT - R;
          ti_ = tc + oi * tpitchT - R;
        }
      } else {  // row lines
        ss = 1;
        so_ = sc + oo * Lt.swp - R;
        si_ = sc + oi * Lt.swp - R;
        const uint32_t *tc;
        int tp;
        if (t.win) {
          tc = s_tgt + (t.ey - toy) * Lt.twp + (t.ex - tox);
          tp = Lt.twp;
        } else {
          tc = tbase + (size_t)t.ph * tpw_ + (size_t)t.ey * tpitch + t.ex;
          tp = tpitch;
        }
        ts = 1;
        to_ = tc + oo * tp - R;
        ti_ = tc + oi * tp - R;
      }
      cost = cq + lane_line_delta<R>(so_, si_, ss, to_, ti_, ts);
    } else {  // one call for both sources, so that a warp never runs the loop twice
      const uint32_t *tc = t.win ? s_tgt + (t.ey - toy) * Lt.twp + (t.ex - tox)
                                 : tbase + (size_t)t.ph * tpw_ + (size_t)t.ey * tpitch + t.ex;
      cost = lane_full<R>(sc, Lt.swp, tc, t.win ? Lt.twp : tpitch);
    }
    return cf;
  };
  auto clamp_flow = [&](int px, int py, uint32_t fq) {
    int X, Y;
    return clamp_target(P.tgt, px, py, fq, X, Y);
  };

  // ---- wavefront over scan anti-diagonals ----
  // Tiles of up to 16 rows: lane j owns scan row j and lane j + 16 evaluates the
  // row's vertical candidate at the same time; larger tiles: lane j owns row j and
  // evaluates both candidates. The owner applies them in order (strict less).
  const bool paired = T <= 16;
  const int row = paired ? (lane & 15) : lane;
  const int role = paired ? (lane >> 4) : 0;
  const int owner = paired ? row : lane;
  uint32_t last_f = 0;
  int32_t last_c = COST_UNSET;
  for (int d = 0; d < tw + th - 1; d++) {
    const uint32_t up_f = __shfl_up_sync(FULL_MASK, last_f, 1, paired ? 16 : 32);
    const int32_t up_c = __shfl_up_sync(FULL_MASK, last_c, 1, paired ? 16 : 32);
    const int jp = row, ip = d - row;
    const bool on = jp < th && ip >= 0 && ip < tw;
    int lx = 0, ly = 0, gx = 0, gy = 0, px = 0, py = 0;
    uint32_t f0 = 0;
    int32_t c0 = COST_UNSET;
    // the sources' states
    bool hv = false, vv = false;
    uint32_t fh = 0, fv = 0;
    int32_t ch = COST_UNSET, cv = COST_UNSET;
    if (on) {
      lx = hdx < 0 ? ip : tw - 1 - ip;
      ly = vdy < 0 ? jp : th - 1 - jp;
      gx = x0 + lx;
      gy = y0 + ly;
      px = gx * n;
      py = gy * n;
      f0 = s_flow[ly * T + lx];
      c0 = s_cost[ly * T + lx];
      if (gx + hdx >= 0 && gx + hdx < Gx) {
        fh = ip > 0 ? last_f : s_hf[ly];
        ch = ip > 0 ? last_c : s_hc[ly];
        hv = ch != COST_UNSET;
      }
      if (gy + vdy >= 0 && gy + vdy < Gy) {
        fv = jp > 0 ? up_f : s_vf[lx];
        cv = jp > 0 ? up_c : s_vc[lx];
        vv = cv != COST_UNSET;
      }
    }
    const bool set = c0 != COST_UNSET;
    uint32_t nf = f0;
    int32_t nc = c0;
    if (paired) {
      // owner: horizontal candidate; helper: vertical candidate (deduplicated
      // against the horizontal one, which would be evaluated first)
      const uint32_t cfh = hv ? clamp_flow(px, py, fh) : 0u;
      const bool useh = hv && !(set && cfh == f0);
      const uint32_t cfv = vv ? clamp_flow(px, py, fv) : 0u;
      const bool usev = vv && !(set && cfv == f0) && !(useh && cfv == cfh);
      int cost = COST_UNSET;
      if (role == 0 && useh) evaluate(0, lx, ly, px, py, fh, ch, cost);
      if (role == 1 && usev) evaluate(1, lx, ly, px, py, fv, cv, cost);
      const int cost_v = __shfl_sync(FULL_MASK, cost, row + 16);
      if (role == 0 && on) {
        if (useh && cost < nc) {
          nc = cost;
          nf = cfh;
        }
        if (usev && cost_v < nc) {
          nc = cost_v;
          nf = cfv;
        }
        s_flow[ly * T + lx] = nf;
        s_cost[ly * T + lx] = nc;
      }
    } else if (on) {
      uint32_t first = 0;
      bool have_first = false;
#pragma unroll
      for (int c = 0; c < 2; c++) {
        const bool ok = c == 0 ? hv : vv;
        if (!ok) continue;
        const uint32_t fq = c == 0 ? fh : fv;
        const uint32_t cf = clamp_flow(px, py, fq);
        if (set && cf == f0) continue;
        if (have_first && cf == first) continue;
        first = cf;
        have_first = true;
        int cost;
        evaluate(c, lx, ly, px, py, fq, c == 0 ? ch : cv, cost);
        if (cost < nc) {
          nc = cost;
          nf = cf;
        }
      }
      s_flow[ly * T + lx] = nf;
      s_cost[ly * T + lx] = nc;
    }
    // the row's last state, identical in the owner and its helper
    const uint32_t lf = on ? nf : last_f;
    const int32_t lc = on ? nc : last_c;
    last_f = __shfl_sync(FULL_MASK, lf, owner);
    last_c = __shfl_sync(FULL_MASK, lc, owner);
  }
  __syncwarp();

  // ---- random search: every lane evaluates the candidates of its own points ----
  if (cfg.do_rs) {
    const int Rn = (cfg.R * n) << P.tgt.log2q;  // offsets in units of 1/q pixel
    for (int i = sl; i < tw * th; i += width) {
      const int lx = i % tw, ly = i / tw;
      const uint32_t cur = s_flow[ly * T + lx];
      const int32_t cc = s_cost[ly * T + lx];
      if (cc == COST_UNSET) continue;
      const int gx = x0 + lx, gy = y0 + ly, px = gx * n, py = gy * n;
      int ox, oy, X, Y;
      rs_offset(cfg.seed, P.flow_id, log2n, cfg.s, gx, gy, Rn, ox, oy);
      const uint32_t cf = clamp_target(P.tgt, px, py, flow_dx(cur) + ox, flow_dy(cur) + oy, X, Y);
      if (cf == cur) continue;
      const Tgt t = locate(px, py, cf);
      if (cfg.evals) count_eval(scnt, true, t.win);
      const uint32_t *sc = s_src + (ly + R + 1) * Lt.swp + (lx + R + 1);
      const uint32_t *tc = t.win ? s_tgt + (t.ey - toy) * Lt.twp + (t.ex - tox)
                                 : tbase + (size_t)t.ph * tpw_ + (size_t)t.ey * tpitch + t.ex;
      const int cost = lane_full<R>(sc, Lt.swp, tc, t.win ? Lt.twp : tpitch);
      if (cost < cc) {
        s_flow[ly * T + lx] = cf;
        s_cost[ly * T + lx] = cost;
      }
    }
    __syncwarp();
  }

  for (int i = sl; i < tw * th; i += width) {
    const int lx = i % tw, ly = i / tw;
    const size_t g = (size_t)(y0 + ly) * Gx + x0 + lx;
    fout[g] = s_flow[ly * T + lx];
    cout[g] = s_cost[ly * T + lx];
  }
  if (cfg.evals) {
    __syncwarp();
    if (lane < 4 && scnt[lane]) atomicAdd(cfg.evals + lane, (unsigned long long)scnt[lane]);
  }
}

// Pass kernel with one CTA per tile (T <= 16): each diagonal step of the
// wavefront is spread over 2 * SPLIT threads per scan row instead of one or two
// lanes. Thread t serves row j = t / (2 SPLIT): the first SPLIT threads of the
// row evaluate its horizontal candidate and the next SPLIT its vertical one, each
// over every SPLIT-th patch line (incremental) or row (full E_d), and the row's
// first thread applies both in order (strict less). Sources are read from the
// tile state in shared memory, one barrier per diagonal. Same schedule and
// results as k_pass.
// SPLIT threads per candidate (2, 4 or 8, an execution parameter): 32 * SPLIT
// threads per CTA.
template <int R, int SPLIT>
__device__ __forceinline__ int part_line_delta(const uint32_t *so_, const uint32_t *si_, int ss,
                                               const uint32_t *to_, const uint32_t *ti_, int ts,
                                               int u) {
  int acc = 0;
#pragma unroll
  for (int k = 0; k < (2 * R + SPLIT) / SPLIT; k++) {
    const int w = u + SPLIT * k;
    if (w <= 2 * R)
      acc += __popc(si_[w * ss] ^ ti_[w * ts]) - __popc(so_[w * ss] ^ to_[w * ts]);
  }
  return acc;
}

template <int R, int SPLIT>
__device__ __forceinline__ int part_full(const uint32_t *sc, int swp, const uint32_t *tc, int tp,
                                         int u) {
  int a0 = 0, a1 = 0;
#pragma unroll
  for (int k = 0; k < (2 * R + SPLIT) / SPLIT; k++) {
    const int v = u + SPLIT * k;
    if (v <= 2 * R) {
      const uint32_t *sr = sc + (v - R) * swp - R, *tr = tc + (v - R) * tp - R;
#pragma unroll
      for (int x = 0; x < 2 * R + 1; x++) {
        const int pc = __popc(sr[x] ^ tr[x]);
        if (x & 1) a1 += pc;
        else a0 += pc;
      }
    }
  }
  return a0 + a1;
}

// Tiles of pass s of problem P (the odd passes' tiles are shifted by T/2).
__device__ __forceinline__ int pass_tiles(const SearchProblem &P, int T, int s) {
  const int off = (s & 1) * (T >> 1);
  return ((P.src.NX + off + T - 1) / T) * ((P.src.NY + off + T - 1) / T);
}

// One tile (index `tile` < pass_tiles) of pass cfg.s of problem P by the whole
// CTA (32 * SPLIT threads); smem holds the tile layout and then four evaluation
// counters. GEN = false is the form for integer flows (q = 1) without evaluation
// counting: the subpixel phase arithmetic and the counters compile away.
template <int R, int SPLIT, bool GEN>
__device__ __forceinline__ void wide_tile(const SearchProblem &P, const PassCfg &cfg, int tile,
                                          uint32_t *smem) {
  constexpr int WIDE_THREADS = 32 * SPLIT;
  const int t = threadIdx.x;
  const int Gx = P.src.NX, Gy = P.src.NY, n = P.src.n, log2n = P.src.log2n;
  const int T = cfg.tile, off = (cfg.s & 1) * (T >> 1);
  const int ntx = (Gx + off + T - 1) / T;
  const int tx = tile % ntx, ty = tile / ntx;
  const int x0 = max(tx * T - off, 0), x1 = min(tx * T - off + T, Gx);
  const int y0 = max(ty * T - off, 0), y1 = min(ty * T - off + T, Gy);
  const int tw = x1 - x0, th = y1 - y0;
  const int hdx = c_pass_src[cfg.s][0][0], vdy = c_pass_src[cfg.s][1][1];
  const TileLayout Lt(T, R);
  const uint32_t *fin = (cfg.s & 1) ? P.flow_b : P.flow_a;
  const int32_t *cin = (cfg.s & 1) ? P.cost_b : P.cost_a;
  uint32_t *fout = (cfg.s & 1) ? P.flow_a : P.flow_b;
  int32_t *cout = (cfg.s & 1) ? P.cost_a : P.cost_b;
  if (cfg.last && P.flow_final) {
    fout = P.flow_final;
    cout = P.cost_final;
  }
  const uint32_t *tbase = P.tgt.base, *tbaseT = P.tgt.baseT;
  const int tpitch = P.tgt.pitch, tpitchT = P.tgt.pitchT;
  const size_t tpw_ = P.tgt.plane_words, tpwT = P.tgt.plane_wordsT;
  const TileSmem S = carve_tile(smem, Lt, T);
  const int lq = GEN ? P.tgt.log2q : 0;         // subpixel phases per axis: 1 << lq
  const bool counting = GEN && cfg.evals != nullptr;
  unsigned *scnt = smem + cfg.words_per_tile;  // evaluation counters (PassCfg::evals)
  if (counting && t < 4) scnt[t] = 0;
  int tox, toy, ph0;
  stage_tile<R>(P, Lt, T, true, x0, y0, x1, y1, hdx, vdy, fin, cin, S, t, WIDE_THREADS, tox, toy,
                ph0);
  __syncthreads();

  // target window hit: the whole patch plus one line inside the staged window
  auto in_win = [&](int ph, int ex, int ey) {
    return ph == ph0 && ex - R - 1 >= tox && ex + R + 1 < tox + Lt.tw && ey - R - 1 >= toy &&
           ey + R + 1 < toy + Lt.tw;
  };
  auto clamp_flow = [&](int px, int py, uint32_t fq) {
    int X, Y;
    return clamp_target_lq(P.tgt, px, py, flow_dx(fq), flow_dy(fq), lq, X, Y);
  };

  // Thread t serves scan row jp = t / (2 SPLIT) (tile row ly), candidate `cand`
  // (0: horizontal source, 1: vertical), part u of it. The row's pixel at diagonal
  // d is ip = d - jp. Its horizontal source is the row's previous pixel, whose
  // result every thread of the row keeps (pf, pc); at ip = 0 it is the staged
  // neighbour outside the tile (cost COST_UNSET where there is none).
  const int jp = t / (2 * SPLIT), cand = (t / SPLIT) & 1, u = t & (SPLIT - 1);
  const bool lead = (t & (2 * SPLIT - 1)) == 0;
  const bool row_on = jp < th;
  const int ly = vdy < 0 ? jp : th - 1 - jp;
  const int py = (y0 + ly) * n;
  uint32_t pf = row_on ? S.hf[ly] : 0u;
  int32_t pc = row_on ? S.hc[ly] : COST_UNSET;
  for (int d = 0; d < tw + th - 1; d++) {
    const int ip = d - jp;
    const bool on = row_on && ip >= 0 && ip < tw;
    int lx = 0, px = 0;
    uint32_t f0 = 0, fh = 0, fv = 0;
    int32_t c0 = COST_UNSET, ch = COST_UNSET, cv = COST_UNSET;
    if (on) {
      lx = hdx < 0 ? ip : tw - 1 - ip;
      px = (x0 + lx) * n;
      f0 = S.flow[ly * T + lx];
      c0 = S.cost[ly * T + lx];
      fh = pf;
      ch = pc;
      // inside the tile, or the staged neighbour above / below it
      fv = jp > 0 ? S.flow[(ly + vdy) * T + lx] : S.vf[lx];
      cv = jp > 0 ? S.cost[(ly + vdy) * T + lx] : S.vc[lx];
    }
    const bool hv = ch != COST_UNSET, vv = cv != COST_UNSET;
    const bool set = c0 != COST_UNSET;
    const uint32_t cfh = hv ? clamp_flow(px, py, fh) : 0u;
    const bool useh = hv && !(set && cfh == f0);
    const uint32_t cfv = vv ? clamp_flow(px, py, fv) : 0u;
    const bool usev = vv && !(set && cfv == f0) && !(useh && cfv == cfh);
    int part = 0;
    if (on && (cand == 0 ? useh : usev)) {
      const uint32_t fq = cand == 0 ? fh : fv, cf = cand == 0 ? cfh : cfv;
      const int32_t cq = cand == 0 ? ch : cv;
      const uint32_t *sc = S.src + (ly + R + 1) * Lt.swp + (lx + R + 1);
      int ph, ex, ey;
      target_plane_lq(P.tgt, (px << lq) + flow_dx(cf), (py << lq) + flow_dy(cf), lq, ph, ex, ey);
      const bool win = in_win(ph, ex, ey);
      if (counting && u == 0) count_eval(scnt, cf != fq, win);
      if (cf == fq) {  // incremental: E(q, f) - outgoing line + incoming line
        // horizontal sources give column lines, vertical ones row lines: `sa`/`ta`
        // step along a line, `sx`/`tx` from one line to the next
        const int step = cand == 0 ? hdx : vdy;
        const int oo = step + step * R, oi = -step * R;
        const int sa = cand == 0 ? Lt.swp : 1, sx = cand == 0 ? 1 : Lt.swp;
        const uint32_t *tb;
        int ta, tx;
        if (win) {
          tb = S.tgt + (ey - toy) * Lt.twp + (ex - tox);
          ta = cand == 0 ? Lt.twp : 1;
          tx = cand == 0 ? 1 : Lt.twp;
        } else if (cand == 0) {  // column lines are rows of the transposed plane
          tb = tbaseT + (size_t)ph * tpwT + (size_t)ex * tpitchT + ey;
          ta = 1;
          tx = tpitchT;
        } else {
          tb = tbase + (size_t)ph * tpw_ + (size_t)ey * tpitch + ex;
          ta = 1;
          tx = tpitch;
        }
        const uint32_t *sb = sc - R * sa;
        tb -= R * ta;
        part = part_line_delta<R, SPLIT>(sb + oo * sx, sb + oi * sx, sa, tb + oo * tx, tb + oi * tx,
                                         ta, u) +
               (u == 0 ? cq : 0);
      } else {  // one call for both sources, so that a warp never runs the loop twice
        const uint32_t *tc = win ? S.tgt + (ey - toy) * Lt.twp + (ex - tox)
                                 : tbase + (size_t)ph * tpw_ + (size_t)ey * tpitch + ex;
        part = part_full<R, SPLIT>(sc, Lt.swp, tc, win ? Lt.twp : tpitch, u);
      }
    }
    // sum over the candidate's SPLIT threads, then swap with the other candidate's
#pragma unroll
    for (int o = 1; o < SPLIT; o <<= 1) part += __shfl_xor_sync(FULL_MASK, part, o);
    const int other = __shfl_xor_sync(FULL_MASK, part, SPLIT);
    const int cost_h = cand == 0 ? part : other, cost_v = cand == 0 ? other : part;
    if (on) {  // every thread of the row applies both candidates, in order
      uint32_t nf = f0;
      int32_t nc = c0;
      if (useh && cost_h < nc) {
        nc = cost_h;
        nf = cfh;
      }
      if (usev && cost_v < nc) {
        nc = cost_v;
        nf = cfv;
      }
      if (lead) {
        S.flow[ly * T + lx] = nf;
        S.cost[ly * T + lx] = nc;
      }
      pf = nf;
      pc = nc;
    }
    __syncthreads();
  }

  if (cfg.do_rs) {  // random search, one thread per point, points row by row
    const int Rn = (cfg.R * n) << lq;  // offsets in units of 1/q pixel
    for (int i = t; i < tw * th; i += WIDE_THREADS) {
      const int lx = i % tw, ly = i / tw;
      const uint32_t cur = S.flow[ly * T + lx];
      const int32_t cc = S.cost[ly * T + lx];
      if (cc == COST_UNSET) continue;
      const int gx = x0 + lx, gy = y0 + ly, px = gx * n, py = gy * n;
      int ox, oy;
      rs_offset(cfg.seed, P.flow_id, log2n, cfg.s, gx, gy, Rn, ox, oy);
      int X, Y;
      const uint32_t cf = clamp_target_lq(P.tgt, px, py, flow_dx(cur) + ox, flow_dy(cur) + oy, lq, X, Y);
      if (cf == cur) continue;
      int ph, ex, ey;
      target_plane_lq(P.tgt, X, Y, lq, ph, ex, ey);
      const uint32_t *sc = S.src + (ly + R + 1) * Lt.swp + (lx + R + 1);
      const bool win = in_win(ph, ex, ey);
      if (counting) count_eval(scnt, true, win);
      // one call for both sources, so that a warp never runs the 289-tap loop twice
      const uint32_t *tc = win ? S.tgt + (ey - toy) * Lt.twp + (ex - tox)
                               : tbase + (size_t)ph * tpw_ + (size_t)ey * tpitch + ex;
      const int cost = lane_full<R>(sc, Lt.swp, tc, win ? Lt.twp : tpitch);
      if (cost < cc) {
        S.flow[ly * T + lx] = cf;
        S.cost[ly * T + lx] = cost;
      }
    }
    __syncthreads();
  }
  for (int i = t; i < tw * th; i += WIDE_THREADS) {
    const int lx = i % tw, ly = i / tw;
    const size_t g = (size_t)(y0 + ly) * Gx + x0 + lx;
    fout[g] = S.flow[ly * T + lx];
    cout[g] = S.cost[ly * T + lx];
  }
  if (counting) {
    __syncthreads();
    if (t < 4 && scnt[t]) atomicAdd(cfg.evals + t, (unsigned long long)scnt[t]);
  }
}

template <int R, int SPLIT, bool GEN>
__global__ void __launch_bounds__(32 * SPLIT, 32 / SPLIT) k_pass_wide(const SearchProblem *probs, PassCfg cfg) {
  extern __shared__ uint32_t smem[];
  const SearchProblem &P = probs[blockIdx.y];
  if ((int)blockIdx.x >= pass_tiles(P, cfg.tile, cfg.s)) return;  // whole CTA
  wide_tile<R, SPLIT, GEN>(P, cfg, blockIdx.x, smem);
}

// ---------------------------------------------------------------------------
// Persistent per-level kernel (batched form): one cooperative launch runs a whole
// hierarchy level for every problem (pair and flow) of a batch: the seeding of
// all problems, then pass 0 .. 3 over a work list of (problem, tile) items (the
// random searches inside the passes), a grid-wide barrier between phases. Items
// are taken in blockIdx order with a grid stride; problems of two patch radii
// RA and RB (the r and r2 flows) share the launch. The tiled schedule and the
// results are those of the per-pass kernels.
struct LevelCfg {
  int nprob;
  const int32_t *tile_base;  // [2][nprob + 1]: prefix sums of the tiles of even / odd passes
  int tile, n_rs, R;
  uint64_t seed;
  int words_per_tile;        // shared words of the larger of the two tile layouts
  int seeded;                // 1: problems are seeded from flow_coarse first
  unsigned *bar;             // grid-barrier arrival counter, zero at launch
  long long budget;          // clock cycles one barrier wait may take
  int skip_block;            // test hook: this block never reaches the first barrier (-1: none)
  DeviceStatus *status;
  unsigned long long *evals_a, *evals_b;  // evaluation counters of radius RA / RB, or nullptr
};

// Grid-wide barrier number k (1-based) of the launch: every CTA adds one to the
// counter and waits until k * gridDim.x arrivals. The wait is bounded by
// lc.budget cycles: when it runs out the CTA raises DEV_ERR_TIMEOUT (block,
// barrier) and gets false, so it can leave. Every thread of the CTA calls it.
__device__ bool grid_barrier(const LevelCfg &lc, int k) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(lc.bar, 1u);
    const unsigned target = (unsigned)k * gridDim.x;
    const long long t0 = clock64();
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(lc.bar) : "memory");
      if (v >= target) break;
      if (clock64() - t0 > lc.budget) {
        ok = 0;
        raise_status(lc.status, DEV_ERR_TIMEOUT, blockIdx.x, k);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Register budget: 85 per thread (6 CTAs of 128 threads or 3 of 256 per SM): the
// two radii's tile paths in one function need more than the per-pass kernels' 64.
template <int RA, int RB, int SPLIT>
__global__ void __launch_bounds__(32 * SPLIT, 24 / SPLIT) k_level(const SearchProblem *probs, LevelCfg lc) {
  extern __shared__ uint32_t smem[];
  int nbar = 0;
  if (lc.seeded) {
    const int l16 = threadIdx.x & 15;
    const unsigned gmask = 0xffffu << (threadIdx.x & 16);
    const int g0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 4, ng = (gridDim.x * blockDim.x) >> 4;
    for (int j = 0; j < lc.nprob; j++) {
      const SearchProblem &P = probs[j];
      const int Gc = seed_blocks(P);
      if (RA == RB || P.r == RA) {
        for (int c = g0; c < Gc; c += ng) seed_block<RA>(P, c, l16, gmask);
      } else {
        for (int c = g0; c < Gc; c += ng) seed_block<RB>(P, c, l16, gmask);
      }
    }
    if ((int)blockIdx.x == lc.skip_block) return;
    if (!grid_barrier(lc, ++nbar)) return;
  }
  for (int s = 0; s < 4; s++) {
    PassCfg cfg{s, lc.tile, (s < 3 && s < lc.n_rs) ? 1 : 0, lc.R, lc.seed, s == 3, lc.words_per_tile,
                nullptr};
    const int32_t *tb = lc.tile_base + (s & 1) * (lc.nprob + 1);
    const int total = tb[lc.nprob];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
      int lo = 0, hi = lc.nprob - 1;  // the problem holding the item: last j with tb[j] <= item
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tb[mid] <= item) lo = mid;
        else hi = mid - 1;
      }
      const SearchProblem &P = probs[lo];
      if (RA == RB || P.r == RA) {
        cfg.evals = lc.evals_a;
        wide_tile<RA, SPLIT, true>(P, cfg, item - tb[lo], smem);
      } else {
        cfg.evals = lc.evals_b;
        wide_tile<RB, SPLIT, true>(P, cfg, item - tb[lo], smem);
      }
      __syncthreads();  // the tile's shared memory is reused by the next item
    }
    if (s < 3) {
      if (!lc.seeded && s == 0 && (int)blockIdx.x == lc.skip_block) return;
      if (!grid_barrier(lc, ++nbar)) return;
    }
  }
}

// One side stream per device, created on first use, lets problems of a second
// patch radius (a separate kernel instantiation) run concurrently with the first:
// fork with an event recorded on the caller's stream, join with one recorded on
// the side stream. Both directions are stream-ordered, so the call stays
// asynchronous and capturable.
struct SideStream {
  cudaStream_t s = nullptr, s2 = nullptr, s3 = nullptr;  // s2, s3: more streams of a SideSection
  cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr, join3 = nullptr;
  cudaEvent_t sig[2] = {nullptr, nullptr};
};
static SideStream g_side[64];
static std::mutex g_side_mu, g_side_enqueue_mu;

static ff_status side_stream(SideStream **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FF_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_side_mu);
  SideStream &S = g_side[dev];
  if (!S.s) {
    if (cudaStreamCreateWithFlags(&S.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S.s2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S.s3, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&S.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&S.join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&S.join2, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&S.join3, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&S.sig[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&S.sig[1], cudaEventDisableTiming) != cudaSuccess)
      return FF_ERR_CUDA;
  }
  *out = &S;
  return FF_OK;
}

// The pass kernel for radius r: k_pass (wide = 0) or k_pass_wide with `wide`
// threads per candidate (2, 4 or 8), in its general form (gen: subpixel flows or
// evaluation counting) or its integer-only form.
static ff_status pass_kernel(int r, int wide, bool gen, const void **fn) {
  *fn = nullptr;
  if (wide == 0) {
    FF_DISPATCH_R(r, *fn = (const void *)k_pass<RR>);
  } else if (gen) {
    if (wide == 2) FF_DISPATCH_R(r, *fn = (const void *)k_pass_wide<RR, 2, true>);
    if (wide == 4) FF_DISPATCH_R(r, *fn = (const void *)k_pass_wide<RR, 4, true>);
    if (wide == 8) FF_DISPATCH_R(r, *fn = (const void *)k_pass_wide<RR, 8, true>);
  } else {
    if (wide == 2) FF_DISPATCH_R(r, *fn = (const void *)k_pass_wide<RR, 2, false>);
    if (wide == 4) FF_DISPATCH_R(r, *fn = (const void *)k_pass_wide<RR, 4, false>);
    if (wide == 8) FF_DISPATCH_R(r, *fn = (const void *)k_pass_wide<RR, 8, false>);
  }
  return *fn ? FF_OK : FF_ERR_INVALID_ARG;
}

// Opt in to more than 48 KB of dynamic shared memory when a tile needs it.
static ff_status set_pass_smem(int r, size_t bytes, int wide, bool gen) {
  const void *fn = nullptr;
  FF_TRY(pass_kernel(r, wide, gen, &fn));
  return smem_opt_in(fn, bytes);
}

// Threads per candidate of k_pass_wide at grid spacing n (execution parameters
// split2_max_n and split8_min_n).
static int pass_split(int n) {
  const int s2 = exec_params().split2_max_n, s8 = exec_params().split8_min_n;
  if (s2 > 0 && n <= s2) return 2;
  return (s8 > 0 && n >= s8) ? 8 : 4;
}

// Multiprocessor count of the current device, looked up once per device.
static ff_status sm_count(int *out) {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FF_ERR_CUDA;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (!v) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
      return FF_ERR_CUDA;
    cache[dev].store(v, std::memory_order_relaxed);
  }
  *out = v;
  return FF_OK;
}

static ff_status launch_group(const SearchProblem *probs, const SearchProblem *d, int np, int r,
                              int tile, int n_rs, int R, uint64_t seed, cudaStream_t st) {
  int maxG = 0, maxT = 0;
  for (int j = 0; j < np; j++) {
    const Planes &S = probs[j].src;
    maxG = max(maxG, S.NX * S.NY);
    const int half = tile / 2;
    maxT = max(maxT, ((S.NX + half + tile - 1) / tile) * ((S.NY + half + tile - 1) / tile));
  }
  int nsm = 0;
  FF_TRY(sm_count(&nsm));
  if (probs[0].flow_coarse) {
    const int blocks = (int)min(((long)(maxG + 3) / 4 * 16 + 255) / 256, (long)nsm * 8);
    dim3 g(max(blocks, 1), np);
    FF_DISPATCH_R(r, k_seed<RR><<<g, 256, 0, st>>>(d));
    FF_CHECK_LAUNCH();
  }
  const TileLayout lay(tile, r);
  const int wide_min_n = exec_params().wide_min_n;
  const bool wide = wide_min_n > 0 && probs[0].src.n >= wide_min_n && tile <= 16;
  const int split = pass_split(probs[0].src.n);
  int pw = exec_params().pass_warps;
  while (pw > 1 && sizeof(uint32_t) * ((size_t)lay.words() + 4) * pw > 227u * 1024u) pw--;
  // a level with few tiles spreads them over the SMs (one CTA per SM at least)
  const long tiles = (long)maxT * np;
  while (pw > 1 && (tiles + pw - 1) / pw < nsm) pw--;
  if (wide) pw = 1;
  // the tiles, then four evaluation counters per warp (k_pass) or per CTA
  const size_t smem = sizeof(uint32_t) * ((size_t)lay.words() * pw + 4 * pw);
  const int log2n = probs[0].src.log2n;
  unsigned long long *evals = prof_evals(r, log2n);
  // the integer-only kernels unless some problem has subpixel flows or the
  // evaluations are counted
  bool gen = evals != nullptr;
  for (int j = 0; j < np; j++) gen = gen || probs[j].tgt.q > 1;
  FF_TRY(set_pass_smem(r, smem, wide ? split : 0, gen));
  const void *fn = nullptr;
  FF_TRY(pass_kernel(r, wide ? split : 0, gen, &fn));
  const dim3 block(wide ? 32 * split : pw * 32);
  const int rs_min_n = exec_params().rs_min_n;
  const bool rs_kernel = rs_min_n > 0 && probs[0].src.n >= rs_min_n;
  for (int s = 0; s < 4; s++) {
    const bool do_rs = s < 3 && s < n_rs;
    PassCfg cfg{s, tile, (do_rs && !rs_kernel) ? 1 : 0, R, seed, s == 3, lay.words(), evals};
    dim3 g((maxT + pw - 1) / pw, np);
    if (prof_enabled()) prof_begin(st, log2n);
    const SearchProblem *dp = d;
    void *args[] = {(void *)&dp, (void *)&cfg};
    (void)cudaLaunchKernel(fn, g, block, args, smem, st);
    FF_CHECK_LAUNCH();
    if (prof_enabled()) prof_end(st);
    if (do_rs && rs_kernel) {
      dim3 gr((maxG * 16 + 255) / 256, np);
      FF_DISPATCH_R(r, k_rs<RR><<<gr, 256, 0, st>>>(d, s, R, seed, evals));
      FF_CHECK_LAUNCH();
    }
  }
  return FF_OK;
}

ff_status SideSection::begin(cudaStream_t st, int nside) {
  g_side_enqueue_mu.lock();
  locked = true;
  SideStream *S = nullptr;
  FF_TRY(side_stream(&S));
  if (nside < 1 || nside > 3) return FF_ERR_INVALID_ARG;
  if (cudaEventRecord(S->fork, st) != cudaSuccess) return FF_ERR_CUDA;
  main = st;
  sig[0] = S->sig[0];
  sig[1] = S->sig[1];
  const cudaStream_t ss[3] = {S->s, S->s2, S->s3};
  const cudaEvent_t js[3] = {S->join, S->join2, S->join3};
  for (int i = 0; i < nside; i++) {
    if (cudaStreamWaitEvent(ss[i], S->fork, 0) != cudaSuccess) return FF_ERR_CUDA;
    side[i] = ss[i];
    join[i] = js[i];
  }
  return FF_OK;
}

ff_status SideSection::signal(int k, cudaStream_t s) {
  if (k < 0 || k > 1 || !sig[k]) return FF_ERR_INVALID_ARG;
  return cudaEventRecord(sig[k], s) == cudaSuccess ? FF_OK : FF_ERR_CUDA;
}

ff_status SideSection::wait(int k, cudaStream_t s) {
  if (k < 0 || k > 1 || !sig[k]) return FF_ERR_INVALID_ARG;
  return cudaStreamWaitEvent(s, sig[k], 0) == cudaSuccess ? FF_OK : FF_ERR_CUDA;
}

ff_status SideSection::end() {
  ff_status r = FF_OK;
  for (int i = 0; i < 3; i++) {
    if (side[i] && (cudaEventRecord(join[i], side[i]) != cudaSuccess ||
                    cudaStreamWaitEvent(main, join[i], 0) != cudaSuccess))
      r = FF_ERR_CUDA;
    side[i] = nullptr;
  }
  if (locked) {
    locked = false;
    g_side_enqueue_mu.unlock();
  }
  return r;
}

// ---------------------------------------------------------- persistent level --
static std::atomic<long long> g_bar_budget{0};
static std::atomic<int> g_bar_skip{-1}, g_net_stall{0};
constexpr long long BAR_BUDGET_DEFAULT = 1ll << 31;  // clock cycles, about a second

void set_wait_test(long long budget_cycles, int skip_block, int net_stall) {
  g_bar_budget.store(budget_cycles);
  g_bar_skip.store(skip_block);
  g_net_stall.store(net_stall);
}
int net_stall_polls() { return g_net_stall.load(); }

// k_level<RA, RB, SPLIT> for one radius (RA == RB, r = 1..8) or the paper's pair
// (8, 6); nullptr for other pairs.
template <int SPLIT>
static const void *level_kernel_split(int ra, int rb) {
  if (ra == rb) {
    switch (ra) {
      case 1: return (const void *)k_level<1, 1, SPLIT>;
      case 2: return (const void *)k_level<2, 2, SPLIT>;
      case 3: return (const void *)k_level<3, 3, SPLIT>;
      case 4: return (const void *)k_level<4, 4, SPLIT>;
      case 5: return (const void *)k_level<5, 5, SPLIT>;
      case 6: return (const void *)k_level<6, 6, SPLIT>;
      case 7: return (const void *)k_level<7, 7, SPLIT>;
      case 8: return (const void *)k_level<8, 8, SPLIT>;
      default: return nullptr;
    }
  }
  if (ra == 8 && rb == 6) return (const void *)k_level<8, 6, SPLIT>;
  return nullptr;
}
static const void *level_kernel(int ra, int rb, int split) {
  return split == 8 ? level_kernel_split<8>(ra, rb) : level_kernel_split<4>(ra, rb);
}

ff_status run_level_persistent(const SearchProblem *probs, SearchProblem *dev, int nprob,
                               int32_t *tile_base, unsigned *bar, DeviceStatus *status, int tile,
                               int n_rs, int R, uint64_t seed, cudaStream_t st) {
  if (nprob <= 0) return FF_OK;
  if (tile > 16 || tile < 2) return FF_ERR_INVALID_ARG;
  int ra = probs[0].r, rb = ra;
  for (int j = 1; j < nprob; j++)
    if (probs[j].r != ra) {
      if (rb != ra && probs[j].r != rb) return FF_ERR_INVALID_ARG;  // at most two radii
      rb = probs[j].r;
    }
  if (ra < rb) std::swap(ra, rb);
  const int log2n = probs[0].src.log2n;
  // the persistent form has 4 or 8 threads per candidate (2 runs as 4)
  const int split = pass_split(probs[0].src.n) == 8 ? 8 : 4;
  const void *fn = level_kernel(ra, rb, split);
  if (!fn) {  // no fused kernel for these two radii: one launch per run of equal radius
    for (int i = 0; i < nprob;) {
      int j = i;
      while (j < nprob && probs[j].r == probs[i].r) j++;
      FF_TRY(run_level_persistent(probs + i, dev + i, j - i, tile_base, bar, status, tile, n_rs, R,
                                  seed, st));
      i = j;
    }
    return FF_OK;
  }
  FF_TRY(upload_desc(probs, dev, nprob, st));
  std::vector<int32_t> tb(2 * (size_t)(nprob + 1));
  for (int par = 0; par < 2; par++) {
    int32_t *b = tb.data() + par * (nprob + 1);
    b[0] = 0;
    for (int j = 0; j < nprob; j++) {
      const int off = par * (tile >> 1);
      b[j + 1] = b[j] + ((probs[j].src.NX + off + tile - 1) / tile) *
                            ((probs[j].src.NY + off + tile - 1) / tile);
    }
  }
  FF_TRY(upload_desc(tb.data(), tile_base, 2 * (nprob + 1), st));
  const int words = max(TileLayout(tile, ra).words(), TileLayout(tile, rb).words());
  const size_t smem = sizeof(uint32_t) * ((size_t)words + 4);
  FF_TRY(smem_opt_in(fn, smem));
  int nsm = 0, occ = 0;
  FF_TRY(sm_count(&nsm));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * split, smem) != cudaSuccess ||
      occ < 1) {
    (void)cudaGetLastError();
    return FF_ERR_CUDA;
  }
  const int items = max(tb[nprob], tb[2 * nprob + 1]);
  const int grid = max(1, min(items, occ * nsm));
  if (cudaMemsetAsync(bar, 0, sizeof(unsigned), st) != cudaSuccess) return FF_ERR_CUDA;
  LevelCfg lc{};
  lc.nprob = nprob;
  lc.tile_base = tile_base;
  lc.tile = tile;
  lc.n_rs = n_rs;
  lc.R = R;
  lc.seed = seed;
  lc.words_per_tile = words;
  lc.seeded = probs[0].flow_coarse != nullptr;
  lc.bar = bar;
  const long long bud = g_bar_budget.load();
  lc.budget = bud > 0 ? bud : BAR_BUDGET_DEFAULT;
  lc.skip_block = g_bar_skip.load();
  lc.status = status;
  lc.evals_a = prof_evals(ra, log2n);
  lc.evals_b = prof_evals(rb, log2n);
  const SearchProblem *dp = dev;
  void *args[] = {(void *)&dp, (void *)&lc};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32 * split);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every block resident: the barriers can complete
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (prof_enabled()) prof_begin(st, log2n);
  if (cudaLaunchKernelExC(&cfg, fn, args) != cudaSuccess) {
    (void)cudaGetLastError();
    return FF_ERR_CUDA;
  }
  count_launch(1);
  if (prof_enabled()) prof_end(st);
  return FF_OK;
}

ff_status run_level_on(const SearchProblem *probs, SearchProblem *dev, int nprob, int tile,
                       int n_rs, int R, uint64_t seed, cudaStream_t st) {
  if (nprob <= 0) return FF_OK;
  for (int i = 1; i < nprob; i++)
    if (probs[i].r != probs[0].r) return FF_ERR_INVALID_ARG;
  FF_TRY(upload_desc(probs, dev, nprob, st));
  return launch_group(probs, dev, nprob, probs[0].r, tile, n_rs, R, seed, st);
}

ff_status run_level(const SearchProblem *probs, SearchProblem *dev, int nprob, int tile, int n_rs,
                    int R, uint64_t seed, cudaStream_t st) {
  if (nprob <= 0) return FF_OK;
  FF_TRY(upload_desc(probs, dev, nprob, st));
  // contiguous runs of equal radius; the first runs on the caller's stream, the
  // others on the side stream concurrently
  int starts[16], counts[16], nruns = 0;
  for (int i = 0; i < nprob;) {
    int j = i;
    while (j < nprob && probs[j].r == probs[i].r) j++;
    if (nruns == 16) return FF_ERR_INVALID_ARG;
    starts[nruns] = i;
    counts[nruns++] = j - i;
    i = j;
  }
  SideStream *side = nullptr;
  // the side stream and its events are shared per device: hold the lock while
  // this call enqueues its fork, launches and join, so calls from several host
  // threads cannot interleave their event records
  std::unique_lock<std::mutex> hold(g_side_enqueue_mu, std::defer_lock);
  if (nruns > 1) {
    hold.lock();
    FF_TRY(side_stream(&side));
    if (cudaEventRecord(side->fork, st) != cudaSuccess ||
        cudaStreamWaitEvent(side->s, side->fork, 0) != cudaSuccess)
      return FF_ERR_CUDA;
  }
  for (int k = 0; k < nruns; k++) {
    cudaStream_t use = (k == 0) ? st : side->s;
    FF_TRY(launch_group(probs + starts[k], dev + starts[k], counts[k], probs[starts[k]].r, tile,
                        n_rs, R, seed, use));
  }
  if (nruns > 1) {
    if (cudaEventRecord(side->join, side->s) != cudaSuccess ||
        cudaStreamWaitEvent(st, side->join, 0) != cudaSuccess)
      return FF_ERR_CUDA;
  }
  return FF_OK;
}

}  // namespace ff
