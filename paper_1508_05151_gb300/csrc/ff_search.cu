// Sec. 3.1 / 3.2: hierarchical propagation (Eq. 2) and random search at one level.
//
// Seeding (level transition): a grid point with both coordinates even takes the
// flow of the coarser level with E_d re-evaluated here; every other point starts
// without a flow (cost 0x7fffffff).
//
// Pass kernel, one CTA per T x T tile of grid points, 512 threads = 32 groups of
// 16 lanes. The fixed parallel schedule: inside the tile the pass is exactly the
// sequential scan (processed as anti-diagonal wavefronts, since a point depends
// only on its left/top -- in scan orientation -- neighbours), and a source
// outside the tile is read from the state at the start of the pass. Odd passes
// shift the tile origin by T/2. Per diagonal:
//   A  warp 0, lane = row: build the point's candidates (its two sources' flows,
//      target clamped into the image), dropping ones equal to the current flow or
//      to the first candidate (they cannot win under strict-less replacement)
//   B  all 32 groups evaluate the candidate list (E_d, 16 lanes per candidate)
//   C  warp 0 applies them in order current, horizontal, vertical (strict less)
// After the wavefront the random search of the pass (if any) runs on all tile
// points in parallel, one group per point.
// The source patches of the tile's points form one dense (T + 2r)^2 block of the
// source frame's phase-(0,0) plane; it is staged in shared memory once per pass.
// Target taps are gathered from the target frame's phase planes (L1/L2).
#include "ff_internal.cuh"

namespace ff {

// Sources of each pass: (dx, dy) of the horizontal, then vertical neighbour.
__constant__ int c_pass_src[4][2][2] = {
    {{-1, 0}, {0, -1}}, {{1, 0}, {0, 1}}, {{1, 0}, {0, -1}}, {{-1, 0}, {0, 1}}};

template <int R>
__global__ void __launch_bounds__(256) k_seed(const SearchProblem *probs) {
  const SearchProblem &P = probs[blockIdx.y];
  const int NX = P.src.NX, G = NX * P.src.NY, n = P.src.n;
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int l16 = threadIdx.x & 15;
  const unsigned gmask = 0xffffu << (threadIdx.x & 16);
  if (g >= G) return;
  const int gx = g % NX, gy = g / NX;
  if ((gx | gy) & 1) {
    if (l16 == 0) {
      P.flow_a[g] = 0;
      P.cost_a[g] = COST_UNSET;
    }
    return;
  }
  const int NXc = (P.src.W + 2 * n - 1) / (2 * n);
  const uint32_t f = P.flow_coarse[(size_t)(gy >> 1) * NXc + (gx >> 1)];
  const int px = gx * n, py = gy * n;
  const int tx = clampi(px + flow_dx(f), 0, P.src.W - 1), ty = clampi(py + flow_dy(f), 0, P.src.H - 1);
  const int cost = group_cost<R>(plane_centre(P.src, px, py), P.src.pitch,
                                 plane_centre(P.tgt, tx, ty), P.tgt.pitch, l16, gmask);
  if (l16 == 0) {
    P.flow_a[g] = pack_flow(tx - px, ty - py);
    P.cost_a[g] = cost;
  }
}

struct PassCfg {
  int s;        // pass 0..3
  int tile;     // T
  int do_rs;    // random search after this pass
  int R;        // full-resolution random-search radius
  uint64_t seed;
  int last;     // last pass of the level (writes flow_final when given)
};

constexpr int PASS_THREADS = 512;
constexpr int NGROUPS = PASS_THREADS / 16;

template <int R>
__global__ void __launch_bounds__(PASS_THREADS) k_pass(const SearchProblem *probs, PassCfg cfg) {
  const SearchProblem &P = probs[blockIdx.y];
  const int Gx = P.src.NX, Gy = P.src.NY, n = P.src.n, W = P.src.W, H = P.src.H;
  const int T = cfg.tile, off = (cfg.s & 1) * (T >> 1);
  const int ntx = (Gx + off + T - 1) / T, nty = (Gy + off + T - 1) / T;
  if ((int)blockIdx.x >= ntx * nty) return;
  const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
  const int x0 = max(tx * T - off, 0), x1 = min(tx * T - off + T, Gx);
  const int y0 = max(ty * T - off, 0), y1 = min(ty * T - off + T, Gy);
  const int tw = x1 - x0, th = y1 - y0;
  const int hdx = c_pass_src[cfg.s][0][0], vdy = c_pass_src[cfg.s][1][1];

  const uint32_t *fin = (cfg.s & 1) ? P.flow_b : P.flow_a;
  const int32_t *cin = (cfg.s & 1) ? P.cost_b : P.cost_a;
  uint32_t *fout = (cfg.s & 1) ? P.flow_a : P.flow_b;
  int32_t *cout = (cfg.s & 1) ? P.cost_a : P.cost_b;
  if (cfg.last && P.flow_final) {
    fout = P.flow_final;
    cout = P.cost_final;
  }

  constexpr int SWP = MAX_TILE + 2 * R;  // staged source window pitch
  __shared__ uint32_t s_src[SWP * SWP];
  __shared__ uint32_t s_flow[MAX_TILE * MAX_TILE];
  __shared__ int32_t s_cost[MAX_TILE * MAX_TILE];
  __shared__ uint32_t s_cflow[2 * MAX_TILE];
  __shared__ int32_t s_cpt[2 * MAX_TILE];
  __shared__ int32_t s_ccost[2 * MAX_TILE];
  __shared__ int s_ncand;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = tid >> 4, l16 = tid & 15;
  const unsigned gmask = 0xffffu << (tid & 16);

  // stage tile state and the source window (phase-(0,0) plane of the source)
  for (int i = tid; i < tw * th; i += PASS_THREADS) {
    const int lx = i % tw, ly = i / tw;
    const size_t g = (size_t)(y0 + ly) * Gx + x0 + lx;
    s_flow[ly * MAX_TILE + lx] = fin[g];
    s_cost[ly * MAX_TILE + lx] = cin[g];
  }
  {
    const uint32_t *src0 = P.src.base + (size_t)(y0 - R + PLANE_PAD) * P.src.pitch + (x0 - R + PLANE_PAD);
    const int ww = tw + 2 * R, wh = th + 2 * R;
    for (int i = tid; i < ww * wh; i += PASS_THREADS) {
      const int wx = i % ww, wy = i / ww;
      s_src[wy * SWP + wx] = src0[(size_t)wy * P.src.pitch + wx];
    }
  }
  __syncthreads();

  // ---- wavefront over anti-diagonals in scan orientation ----
  // lane j of warp 0 owns scan row j' = j; local column from the scan position.
  int my_nc = 0, my_slot = 0;
  uint32_t my_c0 = 0, my_c1 = 0;
  for (int d = 0; d < tw + th - 1; d++) {
    if (warp == 0) {
      // A: candidates of the point on scan row `lane`, scan column d - lane
      const int jp = lane, ip = d - lane;
      int nc = 0;
      uint32_t c0 = 0, c1 = 0;
      const bool on = jp < th && ip >= 0 && ip < tw;
      if (on) {
        const int lx = hdx < 0 ? ip : tw - 1 - ip;
        const int ly = vdy < 0 ? jp : th - 1 - jp;
        const int gx = x0 + lx, gy = y0 + ly, px = gx * n, py = gy * n;
        const uint32_t fcur = s_flow[ly * MAX_TILE + lx];
        const bool set = s_cost[ly * MAX_TILE + lx] != COST_UNSET;
#pragma unroll
        for (int c = 0; c < 2; c++) {
          const int qx = gx + (c == 0 ? hdx : 0), qy = gy + (c == 0 ? 0 : vdy);
          if (qx < 0 || qx >= Gx || qy < 0 || qy >= Gy) continue;
          const int qlx = qx - x0, qly = qy - y0;
          uint32_t fq;
          int32_t cq;
          if (qlx >= 0 && qlx < tw && qly >= 0 && qly < th) {
            fq = s_flow[qly * MAX_TILE + qlx];
            cq = s_cost[qly * MAX_TILE + qlx];
          } else {
            fq = fin[(size_t)qy * Gx + qx];
            cq = cin[(size_t)qy * Gx + qx];
          }
          if (cq == COST_UNSET) continue;
          const int tgx = clampi(px + flow_dx(fq), 0, W - 1), tgy = clampi(py + flow_dy(fq), 0, H - 1);
          const uint32_t cf = pack_flow(tgx - px, tgy - py);
          if (set && cf == fcur) continue;
          if (nc == 1 && cf == c0) continue;
          if (nc == 0) c0 = cf;
          else c1 = cf;
          nc++;
        }
      }
      // slots by exclusive prefix over lanes
      int incl = nc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int slot = incl - nc;
      if (nc > 0) {
        s_cflow[slot] = c0;
        s_cpt[slot] = (jp << 16) | (ip & 0xffff);
        if (nc > 1) {
          s_cflow[slot + 1] = c1;
          s_cpt[slot + 1] = (jp << 16) | (ip & 0xffff);
        }
      }
      if (lane == 31) s_ncand = incl;
      my_nc = nc;
      my_slot = slot;
      my_c0 = c0;
      my_c1 = c1;
    }
    __syncthreads();
    // B: evaluate the candidate list
    const int ncand = s_ncand;
    for (int e = grp; e < ncand; e += NGROUPS) {
      const int jp = s_cpt[e] >> 16, ip = s_cpt[e] & 0xffff;
      const int lx = hdx < 0 ? ip : tw - 1 - ip;
      const int ly = vdy < 0 ? jp : th - 1 - jp;
      const int px = (x0 + lx) * n, py = (y0 + ly) * n;
      const uint32_t cf = s_cflow[e];
      const int cost = group_cost<R>(s_src + (ly + R) * SWP + (lx + R), SWP,
                                     plane_centre(P.tgt, px + flow_dx(cf), py + flow_dy(cf)),
                                     P.tgt.pitch, l16, gmask);
      if (l16 == 0) s_ccost[e] = cost;
    }
    __syncthreads();
    // C: apply in order current, horizontal, vertical
    if (warp == 0 && my_nc > 0) {
      const int jp = lane, ip = d - lane;
      const int lx = hdx < 0 ? ip : tw - 1 - ip;
      const int ly = vdy < 0 ? jp : th - 1 - jp;
      uint32_t f = s_flow[ly * MAX_TILE + lx];
      int32_t c = s_cost[ly * MAX_TILE + lx];
      const int32_t e0 = s_ccost[my_slot];
      if (e0 < c) {
        c = e0;
        f = my_c0;
      }
      if (my_nc > 1) {
        const int32_t e1 = s_ccost[my_slot + 1];
        if (e1 < c) {
          c = e1;
          f = my_c1;
        }
      }
      s_flow[ly * MAX_TILE + lx] = f;
      s_cost[ly * MAX_TILE + lx] = c;
    }
    __syncwarp();
  }
  __syncthreads();

  // ---- random search of this pass: one group per point ----
  if (cfg.do_rs) {
    const int Rn = cfg.R * n;
    for (int i = grp; i < tw * th; i += NGROUPS) {
      const int lx = i % tw, ly = i / tw;
      const uint32_t f = s_flow[ly * MAX_TILE + lx];
      const int32_t c = s_cost[ly * MAX_TILE + lx];
      if (c == COST_UNSET) continue;
      const int gx = x0 + lx, gy = y0 + ly, px = gx * n, py = gy * n;
      int ox, oy;
      rs_offset(cfg.seed, P.flow_id, P.src.log2n, cfg.s, gx, gy, Rn, ox, oy);
      const int tgx = clampi(px + flow_dx(f) + ox, 0, W - 1), tgy = clampi(py + flow_dy(f) + oy, 0, H - 1);
      const uint32_t cf = pack_flow(tgx - px, tgy - py);
      if (cf == f) continue;
      const int cost = group_cost<R>(s_src + (ly + R) * SWP + (lx + R), SWP,
                                     plane_centre(P.tgt, tgx, tgy), P.tgt.pitch, l16, gmask);
      if (l16 == 0 && cost < c) {
        s_flow[ly * MAX_TILE + lx] = cf;
        s_cost[ly * MAX_TILE + lx] = cost;
      }
    }
    __syncthreads();
  }

  for (int i = tid; i < tw * th; i += PASS_THREADS) {
    const int lx = i % tw, ly = i / tw;
    const size_t g = (size_t)(y0 + ly) * Gx + x0 + lx;
    fout[g] = s_flow[ly * MAX_TILE + lx];
    cout[g] = s_cost[ly * MAX_TILE + lx];
  }
}

ff_status run_level(const SearchProblem *probs, SearchProblem *dev, int nprob, int tile, int n_rs,
                    int R, uint64_t seed, cudaStream_t st) {
  if (nprob <= 0) return FF_OK;
  FF_TRY(upload_desc(probs, dev, nprob, st));
  // problems with different radii run as separate launches of the same kernels
  int radii[8], nr = 0;
  for (int i = 0; i < nprob; i++) {
    bool seen = false;
    for (int k = 0; k < nr; k++) seen |= radii[k] == probs[i].r;
    if (!seen) radii[nr++] = probs[i].r;
  }
  for (int k = 0; k < nr; k++) {
    const int r = radii[k];
    // contiguous runs of problems with this radius
    for (int i = 0; i < nprob;) {
      if (probs[i].r != r) {
        i++;
        continue;
      }
      int j = i;
      int maxG = 0, maxT = 0;
      while (j < nprob && probs[j].r == r) {
        const Planes &S = probs[j].src;
        maxG = max(maxG, S.NX * S.NY);
        const int half = tile / 2;
        maxT = max(maxT, ((S.NX + half + tile - 1) / tile) * ((S.NY + half + tile - 1) / tile));
        j++;
      }
      const SearchProblem *d = dev + i;
      const int np = j - i;
      if (probs[i].flow_coarse) {
        dim3 g((maxG * 16 + 255) / 256, np);
        FF_DISPATCH_R(r, k_seed<RR><<<g, 256, 0, st>>>(d));
        FF_CHECK_LAUNCH();
      }
      for (int s = 0; s < 4; s++) {
        PassCfg cfg{s, tile, (s < 3 && s < n_rs) ? 1 : 0, R, seed, s == 3};
        dim3 g(maxT, np);
        if (prof_enabled()) prof_begin(st);
        FF_DISPATCH_R(r, k_pass<RR><<<g, PASS_THREADS, 0, st>>>(d, cfg));
        FF_CHECK_LAUNCH();
        if (prof_enabled()) prof_end(st);
      }
      i = j;
    }
  }
  return FF_OK;
}

}  // namespace ff
