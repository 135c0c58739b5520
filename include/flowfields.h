/*
 * flowfields.h -- C ABI of the GB300 Flow Fields library (libflowfields.so).
 *
 * Flow Fields: dense correspondence fields for large displacement optical flow
 * (Bailer, Taetz, Stricker, ICCV 2015). The library computes, for a pair of 8-bit
 * RGB images, the forward flow field and two backward flow fields by kd-tree
 * initialisation and hierarchical propagation with random search (Sec. 3.1,
 * 3.2), then removes outliers with the two-way consistency check and the region
 * filter (Sec. 3.4) and sparsifies the result (Sec. 3.5). Interpolation of the
 * sparse matches (EpicFlow) is not part of it.
 *
 * Conventions shared by every entry point
 *   - Every pointer argument is DEVICE memory owned by the caller, unless the
 *     description says otherwise. The library allocates no device memory; the
 *     scratch it needs comes from the caller's workspace `ws` of `ws_bytes`
 *     bytes (256-byte aligned), sized by the matching *_workspace_size call.
 *   - Images are uint8, H x W x 3 (RGB), rows tightly packed.
 *   - Flows are int16 pairs (dx, dy), interleaved, in full-resolution pixels;
 *     the target of pixel p is p + flow and always lies inside the image.
 *     A level-n flow field has one entry per grid point (n*gx, n*gy),
 *     Gx = ceil(W/n) by Gy = ceil(H/n), row major.
 *   - Costs are int32 E_d values; 0x7fffffff marks a grid point without a flow.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Every call
 *     enqueues its work on it and returns without synchronising.
 *   - Arguments are checked on the host before anything is enqueued; a failed
 *     check returns an error and enqueues nothing. FF_ERR_CUDA reports a failed
 *     launch. Nothing is thrown across this boundary.
 *   - Results are a pure function of the inputs and ff_params; they do not
 *     depend on streams, batch composition or execution tuning.
 */
#ifndef FLOWFIELDS_H
#define FLOWFIELDS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FF_OK = 0,
  FF_ERR_INVALID_ARG = 1, /* null pointer or parameter out of range */
  FF_ERR_SHAPE = 2,       /* image size outside the supported range */
  FF_ERR_WORKSPACE = 3,   /* workspace missing, misaligned or too small */
  FF_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed */
  FF_ERR_DEVICE = 5       /* a device-side check failed (see ff_device_status) */
} ff_status;

/* Method parameters (Sec. 4 gives k=3, R=1, l=8, r=8, r2=6 and eps/e/s per
 * dataset). tile is the tile edge T of the fixed parallel propagation schedule:
 * grid points are processed in T x T tiles, sequentially inside a tile and from
 * the start-of-pass state across tile borders; odd passes shift the tiles by
 * T/2. T changes results (it is part of the method's definition here), the
 * CUDA launch shapes do not. */
typedef struct ff_params {
  int32_t k;    /* hierarchy levels; the coarsest grid has spacing 2^k (0..4) */
  int32_t r;    /* patch radius of the forward and first backward flow (1..8) */
  int32_t r2;   /* patch radius of the second backward flow (1..8) */
  int32_t leaf; /* kd-tree leaf size l (2..32) */
  int32_t R;    /* random-search radius at full resolution; R_n = R*n (0..64) */
  int32_t eps;  /* consistency threshold eps of Eq. 5, in pixels (1..1000) */
  int32_t e;    /* minimum surviving pixels per 3x3 block (Sec. 3.5) (1..9) */
  int32_t s;    /* region-size threshold of the region filter (Sec. 3.4) (>= 0) */
  int32_t tile; /* tile edge T of the parallel schedule (even, 2..32) */
  int32_t n_rs; /* random-search steps per level, after passes 0..n_rs-1 (0..3) */
  int32_t K;    /* proposals per coarsest grid point for the forward flow (0..8) */
  int32_t color; /* 0: the input RGB channels; 1: integer CIELab (ff_rgb_to_lab) of
                    both frames before every other step (Sec. 3.1, 3.3) */
  int32_t subpel; /* 1, 2 or 4: flows in units of 1/subpel pixel. With 2 or 4 the
                    random search draws subpixel offsets and every subpixel target
                    reads the census of the target frame interpolated there
                    (bilinear colours, Sec. 3.1), exactly in integers; the filter's
                    thresholds scale likewise (ff_flow_fields / _batch / graphs;
                    the per-level entry points take subpel = 1) */
  uint64_t seed; /* seed of the counter-based random search */
} ff_params;

enum { FF_PRESET_SINTEL = 0, FF_PRESET_MIDDLEBURY = 1, FF_PRESET_KITTI = 2 };

/* Human-readable name of a status code (static string). */
const char *ff_status_str(ff_status s);

/* Fill *p with the parameters of Sec. 4 for a dataset preset: k=3, R=1, l=8,
 * r=8, r2=6 and (eps, e, s) = (5, 4, 50) Sintel, (1, 7, 50) Middlebury,
 * (1, 9, 150) KITTI; tile=16, n_rs=3, K=0, seed=0. */
ff_status ff_params_preset(ff_params *p, int preset);

/* Workspace bytes needed by ff_flow_fields for a W x H pair (host-only call). */
ff_status ff_workspace_size(int W, int H, const ff_params *p, size_t *bytes);

/* Sec. 3.1 / 3.3: the paper computes WHT features and census in CIELab. Integer
 * CIELab of an 8-bit sRGB image (D65 white, IEC 61966-2-1 primaries), exact
 * after a 256-entry decoding table lin = round(65536 g(v/255)) (g the sRGB
 * decoding curve): t = (row . lin + 8192) >> 14 with the white-normalised
 * sRGB->XYZ rows in Q14 (each summing to 16384); f(t) = the largest y with
 * y^3 <= t * 2^32 when t * 29^3 > 6^3 * 65536, else (29*841*t + 108*4*65536 +
 * 1566) / 3132; out = (L * 255/100, a + 128, b + 128) with L = 116 f_Y - 16,
 * a = 500 (f_X - f_Y), b = 200 (f_Y - f_Z) in units of 65536, rounded half up
 * and clamped to [0, 255]. img, out: H x W x 3 uint8 (device). */
ff_status ff_rgb_to_lab(const uint8_t *img, int W, int H, uint8_t *out, void *stream);

/* Sec. 3.2: the smoothed full-resolution image I^n: area downsampling by n
 * (block mean, (sum + cnt/2) / cnt over the in-image part of each block),
 * then separable Lanczos-3 upsampling back to W x H with Q14 weights (the
 * coarse sample j is centred on pixel j*n + (n-1)/2; horizontal pass kept
 * unrounded, vertical pass rounded (acc + 2^27) >> 28 and clamped to [0,255]).
 * n is a power of two 1..16; n = 1 copies. img, out: W x H x 3. The workspace
 * holds the coarse image and the horizontal pass (ff_smooth_workspace_size). */
ff_status ff_smooth_workspace_size(int W, int H, int n, size_t *bytes);
ff_status ff_smooth(const uint8_t *img, int W, int H, int n, uint8_t *out, void *ws,
                    size_t ws_bytes, void *stream);

/* Sec. 3.3: census transform of I^n with neighbour spacing n: bit 8c+o is set
 * when channel c of the o-th neighbour (raster order of the 3x3 neighbourhood,
 * centre skipped, coordinates clamped) is below the centre. out: H x W uint32. */
ff_status ff_census(const uint8_t *img_n, int W, int H, int n, uint32_t *out, void *stream);

/* Sec. 3.1: Walsh-Hadamard features of the (2r+1)^2 patch around each pixel:
 * the window is split r | r+1 and again into 4 blocks per axis; the first three
 * Walsh functions in sequency order ((++++), (++--), (+--+)) per axis give 9
 * bases per channel, feature 9c + 3i + j with i the row function. Pixels are
 * read with clamped coordinates; r is 1..8. pts (x, y int32 pairs, npts of them) selects
 * the pixels; pts = NULL computes every pixel in raster order (npts ignored).
 * feat: int32 rows of 28 (27 features + one zero pad), one row per pixel. */
ff_status ff_features(const uint8_t *img, int W, int H, int r, const int32_t *pts, int npts,
                      int32_t *feat, void *stream);

/* Depth D of the kd tree over N points with leaf size `leaf` (the smallest d
 * with ceil(N / 2^d) <= leaf) and the workspace ff_kdtree_build needs. Host. */
ff_status ff_kdtree_size(int N, int leaf, int *depth, size_t *ws_bytes);

/* Sec. 3.1: kd tree over feature rows feat[N][28] (as written by ff_features).
 * Every node splits in the dimension of largest (max - min), lowest index on
 * ties, at the median: the first floor(m/2) of its m points under the order
 * (value, pixel index) go left, and the split value is the value of the first
 * point on the right. Outputs, heap order (children of node i are 2i+1, 2i+2):
 * split_dim[2^D - 1], split_val[2^D - 1]; perm[N] lists the point indices leaf
 * by leaf, leaf j holding positions obtained by halving [0, N) along its path
 * (the left half takes floor(m/2)). The order inside a leaf is unspecified. */
ff_status ff_kdtree_build(const int32_t *feat, int N, int leaf, int32_t *perm, int32_t *split_dim,
                          int32_t *split_val, void *ws, size_t ws_bytes, void *stream);

/* Eq. 1 / Eq. 4: initial flow at the grid of spacing n. For each grid point
 * its WHT vector (features of src_img at radius r) descends the tree built over
 * the W*H target pixels (no backtracking: left iff value < split value); every
 * pixel of the reached leaf is a candidate, and the one with the smallest E_d on
 * P^n_r wins, ties to the lowest pixel index. Then the K proposals of the point
 * (int16 pairs, [Gy][Gx][K][2], NULL when K = 0) are tried in order; a candidate
 * replaces the current flow only when its E_d is strictly lower. Targets are
 * clamped into the image. census_src / census_tgt: level-n census (H x W).
 * A split dimension outside [0, 27) or a perm entry outside [0, W*H) is not
 * dereferenced: it sets device status code 1 (ff_device_status).
 * Outputs flow [Gy][Gx][2], cost [Gy][Gx]. Workspace: ff_level_workspace_size. */
ff_status ff_kdtree_init(const int32_t *perm, const int32_t *split_dim, const int32_t *split_val,
                         int leaf, const uint8_t *src_img, const uint32_t *census_src,
                         const uint32_t *census_tgt, int W, int H, int n, int r,
                         const int16_t *proposals, int K, int16_t *flow, int32_t *cost, void *ws,
                         size_t ws_bytes, void *stream);

/* Workspace bytes of ff_search_level / ff_kdtree_init at spacing n (host). */
ff_status ff_level_workspace_size(int W, int H, int n, size_t *bytes);

/* Sec. 3.1 / 3.2: one hierarchy level at spacing n with patch radius r.
 * If flow_coarse (level 2n, [ceil(H/2n)][ceil(W/2n)][2]) is given, grid points
 * with both coordinates even take the coarse flow with E_d re-evaluated at this
 * level and all others start without a flow; if it is NULL, (flow, cost) hold
 * the initial state on entry. Then four propagation passes (Eq. 2), sources
 * (x-n,y),(x,y-n) / (x+n,y),(x,y+n) / (x+n,y),(x,y-n) / (x-n,y),(x,y+n), each
 * pass scanning away from its sources in the tiled schedule of ff_params.tile,
 * and after passes 0..n_rs-1 a random search with an offset uniform in
 * [-R*n, R*n]^2 drawn from SplitMix64 of (seed, flow_id, log2 n, step, gx, gy).
 * A candidate wins only with strictly lower E_d; targets are clamped into the
 * image. flow_id (0..3) separates the random streams of the three flows.
 * Outputs flow [Gy][Gx][2] and cost [Gy][Gx] at this level. */
ff_status ff_search_level(const uint32_t *census_src, const uint32_t *census_tgt, int W, int H,
                          int n, int r, const int16_t *flow_coarse, const ff_params *p,
                          int flow_id, int16_t *flow, int32_t *cost, void *ws, size_t ws_bytes,
                          void *stream);

/* Sec. 3.4 / 3.5: outlier filtering of the forward flow F against the backward
 * flows Fb1 (radius r) and Fb2 (radius r2), all H x W x 2.
 *   Eq. 5: e_j = |F(p) + Fb_j(p + F(p))|^2; the pixel passes when e_1 and e_2 are
 *          both below eps^2; err_sum = e_1 + e_2 (squared errors; a diagnostic
 *          output: INT32_MAX for a target outside the image).
 *   Region filter: passing pixels whose 4-neighbours differ in flow by less than
 *          3 px form regions; a region of fewer than s pixels is removed when one
 *          of its pixels has a 4-neighbour rejected by Eq. 5 whose flow is within
 *          3 px of it. Result: valid [H][W] (0/1).
 *   Sparsification: in each aligned 3x3 block with at least e valid pixels the
 *          one whose two consistency errors sum to the least, sqrt(e_1) +
 *          sqrt(e_2) compared exactly (first in raster order on ties), is kept:
 *          mask [H][W] and rows (x, y, dx, dy) int32 in block raster order in
 *          sparse [ceil(W/3)*ceil(H/3)][4]; *n_sparse (device int32) = row count.
 * Workspace: ff_filter_workspace_size. */
ff_status ff_filter_workspace_size(int W, int H, size_t *bytes);
ff_status ff_consistency_filter(const int16_t *F, const int16_t *Fb1, const int16_t *Fb2, int W,
                                int H, const ff_params *p, uint8_t *valid, int32_t *err_sum,
                                int32_t *sparse, int32_t *n_sparse, uint8_t *mask, void *ws,
                                size_t ws_bytes, void *stream);

/* Allocation-free variant of ff_consistency_filter (the paper has no
 * counterpart; this exists for callers that cannot allocate device memory).
 * Some callers cannot provide a workspace: a plugin running inside a framework
 * that owns the whole device memory pool and exposes no allocator, or a
 * real-time frame loop that reserves all memory at start-up and must not call
 * cudaMalloc afterwards (it can synchronise the device and stall the loop).
 * This call needs no workspace: its scratch is one static device array of
 * 12 MiB inside the library, which every GPU that loads the library keeps until
 * the process exits. Limits and behaviour:
 *   - W * H <= 1,048,576 pixels; larger images return FF_ERR_SHAPE and enqueue
 *     nothing. Inputs, outputs and results are exactly those of
 *     ff_consistency_filter.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call shares the one array and the array keeps the last call's
 *     contents (the call clears what must start at zero itself): calls whose
 *     work overlaps on the GPU (different streams, or several host threads)
 *     race and corrupt each other's results. Serialise them, e.g. on one stream. */
ff_status ff_consistency_filter_static(const int16_t *F, const int16_t *Fb1, const int16_t *Fb2,
                                       int W, int H, const ff_params *p, uint8_t *valid,
                                       int32_t *err_sum, int32_t *sparse, int32_t *n_sparse,
                                       uint8_t *mask, void *stream);

/* Sec. 4.1 (Table 1, "k=3+median"): the raw forward field filtered by a median
 * weighted by the matching error (the paper gives neither window nor weights;
 * this is the library's reading). E(p) = E_d of pixel p's own flow at full
 * resolution (census of I1 and I2 with spacing 1, patch radius r, taps clamped);
 * weight w(q) = floor(65536 / (1 + E(q))); window: the in-image pixels q with
 * max(|qx - px|, |qy - py|) <= rho (0..3); each component of out(p) is the
 * smallest value v whose samples <= v carry at least half of the window's total
 * weight. I1, I2: H x W x 3; flow, out: int16 [H][W][2] (out != flow);
 * match_err: NULL or int32 [H][W] receiving E. ws: ff_median_workspace_size. */
ff_status ff_median_workspace_size(int W, int H, size_t *bytes);
ff_status ff_weighted_median(const uint8_t *I1, const uint8_t *I2, const int16_t *flow, int W,
                             int H, int r, int rho, int16_t *out, int32_t *match_err, void *ws,
                             size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Sec. 3.3, the second data term: SIFT flow (used by the paper for KITTI, Sec. 5,
 * with r = 3, r2 = 2 and S = 12, S2 = 18 colour channels). Each pixel gets a
 * 128-D SIFT vector, reduced by PCA to S "SIFT flow colours"; E_d sums the L2
 * distance of the colours over the patch taps; the images I^n are the colours
 * smoothed like the frames (Sec. 3.2). The paper names the descriptor only; the
 * library's reading, exact in integers:
 *   - grey g = R + G + B; gx = g(x+1, y) - g(x-1, y), gy likewise (clamped);
 *   - 8 orientations: o_k = max(0, gx C_k + gy S_k), (C_k, S_k) = 256 (cos, sin)
 *     of k * 45 degrees (x right, y down), 1/sqrt 2 as 181/256;
 *   - 4 x 4 cells of 3 x 3 pixels: cell (i, j) sums o_k over x in
 *     [px + 3 (i - 2), px + 3 (i - 1)), y likewise with j (clamped); element
 *     d = (4 j + i) 8 + k;
 *   - normalisation (unit length, clip at 0.2, unit length, x 512, clamp 255) in
 *     integers: N2 = sum h^2, t = isqrt(N2 / 25), h' = min(h, t), M2 = sum h'^2,
 *     q = min(255, isqrt(2^18 h'^2 / M2)), 0 when M2 = 0.
 * ------------------------------------------------------------------------- */

/* Dense SIFT vectors of an RGB frame. img: H x W x 3; desc: uint8 [H][W][128]
 * (16-byte aligned). */
ff_status ff_sift_descriptors(const uint8_t *img, int W, int H, uint8_t *desc, void *stream);

/* PCA statistics of N descriptors (desc: uint8 [N][128], 16-byte aligned), ADDED
 * to sum (uint64 [128]: sum of q_i) and gram (uint64 [128][128]: sum of q_i q_j),
 * exactly; the caller zeroes them before the first call. N < 2^31. */
ff_status ff_sift_moments(const uint8_t *desc, int N, uint64_t *sum, uint64_t *gram,
                          void *stream);

/* The PCA basis of Sec. 3.3 from the statistics of `count` descriptors (count is a
 * host value). Covariance C = gram / count - mu mu^T in float64 (mu = sum / count);
 * its eigenvectors by cyclic Jacobi rotations (round-robin order), sorted by
 * eigenvalue, largest first (ties: lower index), each signed so that its entry
 * of largest magnitude (lowest index on ties) is positive. One gain for all
 * components, g = 127 / (3 sqrt(max(lambda_1, 1))), keeps colour distances
 * proportional to descriptor distances. Outputs (device): basis int16 [S][128],
 * B_si = clamp(floor(4096 g e_si + 1/2), -32767, 32767); offset int32 [S],
 * o_s = 2048 - round_half_up(sum_i B_si sum_i / count) (exact); eigval float64
 * [128] (descending; may be NULL). S is 3..30, a multiple of 3. Device status 3
 * (ff_device_status) if the rotations have not converged after 40 sweeps.
 * ws: ff_sift_pca_workspace_size. */
ff_status ff_sift_pca_workspace_size(size_t *bytes);
ff_status ff_sift_pca(const uint64_t *sum, const uint64_t *gram, int64_t count, int S,
                      int16_t *basis, int32_t *offset, double *eigval, void *ws, size_t ws_bytes,
                      void *stream);

/* SIFT flow colours: channel s of pixel p is clamp(128 + floor((sum_i B_si q_i +
 * o_s) / 4096), 0, 255), stored in S/3 groups of three channels, each group an
 * H x W x 3 image: colors[(s/3)][y][x][s%3] (so ff_smooth gives I^n per group).
 * desc: uint8 [H][W][128]; basis, offset as ff_sift_pca writes them. */
ff_status ff_sift_colors(const uint8_t *desc, int W, int H, const int16_t *basis,
                         const int32_t *offset, int S, uint8_t *colors, void *stream);

/* The kd initialisation (as ff_kdtree_init, K = 0) and one hierarchy level (as
 * ff_search_level) with the SIFT flow data term: E_d = sum over the (2r+1)^2
 * taps of P^n_r (clamped) of floor(16 |c_src - c_tgt|_2), the colours taken
 * from colors_src / colors_tgt (level-n colour groups, S/3 x H x W x 3, as
 * ff_sift_colors writes them after ff_smooth per group). The kd tree is built
 * over WHT features as for the census path. ws: ff_sift_level_workspace_size. */
ff_status ff_sift_level_workspace_size(int W, int H, int n, int S, size_t *bytes);
ff_status ff_sift_kdtree_init(const int32_t *perm, const int32_t *split_dim,
                              const int32_t *split_val, int leaf, const uint8_t *src_img,
                              const uint8_t *colors_src, const uint8_t *colors_tgt, int S, int W,
                              int H, int n, int r, int16_t *flow, int32_t *cost, void *ws,
                              size_t ws_bytes, void *stream);
ff_status ff_sift_search_level(const uint8_t *colors_src, const uint8_t *colors_tgt, int S, int W,
                               int H, int n, int r, const int16_t *flow_coarse, const ff_params *p,
                               int flow_id, int16_t *flow, int32_t *cost, void *ws,
                               size_t ws_bytes, void *stream);

/* The whole path of ff_flow_fields with the SIFT flow data term: SIFT vectors of
 * both input frames; colours with (basis1, offset1, S1) for the forward and the
 * first backward flow and with (basis2, offset2, S2) for the second backward
 * flow (radius r2); per level every colour group smoothed like I^n; kd trees over
 * WHT features (CIELab when p->color = 1); then ff_consistency_filter. Integer
 * flows only (p->subpel must be 1) and no proposals (p->K is ignored). Outputs as
 * ff_flow_fields. ws: ff_sift_workspace_size. */
ff_status ff_sift_workspace_size(int W, int H, const ff_params *p, int S1, int S2, size_t *bytes);
ff_status ff_sift_flow_fields(const uint8_t *I1, const uint8_t *I2, int W, int H,
                              const ff_params *p, const int16_t *basis1, const int32_t *offset1,
                              int S1, const int16_t *basis2, const int32_t *offset2, int S2,
                              int16_t *flows, uint8_t *valid, int32_t *err_sum, int32_t *sparse,
                              int32_t *n_sparse, uint8_t *mask, void *ws, size_t ws_bytes,
                              void *stream);

/* The whole path for one pair (Fig. 2): smoothed images and census for both
 * frames at every level, three flow fields (forward I1->I2 with r, backward
 * I2->I1 with r and with r2; flow ids 0, 1, 2), each from its own kd tree, then
 * ff_consistency_filter. proposals: NULL or int16 [ceil(H/2^k)][ceil(W/2^k)][K][2]
 * for the forward flow. Outputs: flows [3][H][W][2], valid, err_sum, sparse,
 * n_sparse (device int32), mask as in ff_consistency_filter. */
ff_status ff_flow_fields(const uint8_t *I1, const uint8_t *I2, int W, int H, const ff_params *p,
                         const int16_t *proposals, int16_t *flows, uint8_t *valid,
                         int32_t *err_sum, int32_t *sparse, int32_t *n_sparse, uint8_t *mask,
                         void *ws, size_t ws_bytes, void *stream);

/* Batched form (not in the paper): many pairs, possibly of different sizes, in
 * one call. Each pair's results equal those of ff_flow_fields on that pair. The
 * per-image steps run per pair; the kd builds, kd queries and every propagation
 * pass of one flow take that flow's problems of all pairs in the same launches,
 * the three flows on streams of their own (joined back into `stream` before the
 * call's last work, so the call stays stream-ordered). The ff_pair array
 * is host memory; its buffers are device memory as in ff_flow_fields. */
#define FF_MAX_BATCH 256
typedef struct ff_pair {
  const uint8_t *I1, *I2; /* H x W x 3 */
  int W, H;
  const int16_t *proposals; /* NULL or as in ff_flow_fields */
  int16_t *flows;           /* [3][H][W][2] */
  uint8_t *valid;           /* [H][W] */
  int32_t *err_sum;         /* [H][W] */
  int32_t *sparse;          /* [ceil(W/3)*ceil(H/3)][4] */
  int32_t *n_sparse;        /* device int32 */
  uint8_t *mask;            /* [H][W] */
} ff_pair;
ff_status ff_batch_workspace_size(int npairs, const ff_pair *pairs, const ff_params *p,
                                  size_t *bytes);
ff_status ff_flow_fields_batch(int npairs, const ff_pair *pairs, const ff_params *p, void *ws,
                               size_t ws_bytes, void *stream);

/* CUDA graph of one batch: captures the launches of ff_flow_fields_batch for
 * these pairs, buffers and workspace (on `stream`, which must not be the legacy
 * default stream) and instantiates them once; ff_graph_launch replays the whole
 * batch with one call. The buffers' contents may change between launches, their
 * addresses may not. ff_graph_kernel_count gives the kernels one launch runs. */
typedef struct ff_graph ff_graph;
ff_status ff_graph_create(int npairs, const ff_pair *pairs, const ff_params *p, void *ws,
                          size_t ws_bytes, void *stream, ff_graph **out);
ff_status ff_graph_launch(ff_graph *g, void *stream);
ff_status ff_graph_kernel_count(const ff_graph *g, uint64_t *kernels);
ff_status ff_graph_destroy(ff_graph *g);

/* Execution parameters: launch shapes that change speed but never results
 * (the autotuner in the Python package picks them per GPU and workload).
 * Process-wide; set them between calls, not while work is being enqueued.
 *   pass_warps  most tiles (one warp each) per CTA of the propagation kernel,
 *               1..8; a level with few tiles uses fewer so that its CTAs
 *               cover the SMs
 *   rs_min_n    0: every random search runs inside the propagation kernel on
 *               the tile's shared-memory state; else levels with spacing
 *               n >= rs_min_n (a power of two, 1..128) run it as a separate
 *               kernel with one 16-lane group per grid point. Each point's
 *               random search depends only on its own state after the pass,
 *               so both forms give the same result.
 *   wide_min_n  0: every level runs the propagation with one warp per tile; else
 *               levels with spacing n >= wide_min_n (a power of two, 1..128; only
 *               for tiles of edge <= 16) run it with one CTA per tile and
 *               8 threads per scan row (same schedule, same results)
 *   split8_min_n  0: that form uses 4 threads per candidate (128-thread CTAs);
 *               else levels with n >= split8_min_n (a power of two, 1..128) use 8
 *               (256-thread CTAs, 16 threads per scan row)
 *   split2_max_n  0: as above; else levels with n <= split2_max_n (a power of
 *               two, 1..128) use 2 threads per candidate (64-thread CTAs, 4
 *               threads per scan row); takes precedence over split8_min_n
 *   serial_flows  0: the three flows of a pair and the image pyramid run on
 *               four streams concurrently; 1: all on the caller's stream, one
 *               after another (so that one kernel can be timed alone)
 *   kd_merge    0: each flow builds its kd trees on its own stream; 1: the trees
 *               of all flows are built in one launch chain (every launch over
 *               all trees) before the flows fork
 *   persist_levels  0: every level runs a seeding launch and four pass launches
 *               per flow; 1 (tiles of edge <= 16): one persistent cooperative
 *               launch per level runs the seeding and all four passes of every
 *               pair and flow, over a work list of (pair, flow, tile) items,
 *               with a grid-wide barrier between the phases whose wait is
 *               bounded (a wait that runs out sets device status code 3 and the
 *               launch returns; ff_device_status reports it) */
typedef struct ff_exec_params {
  int32_t pass_warps;
  int32_t rs_min_n;
  int32_t wide_min_n;
  int32_t split8_min_n;
  int32_t serial_flows;
  int32_t kd_merge;
  int32_t persist_levels;
  int32_t split2_max_n;
} ff_exec_params;
ff_status ff_set_exec_params(const ff_exec_params *e);
/* Test hooks of the bounded waits (not in the paper); they exist to test the
 * timeout paths without faulting the GPU. Process-wide, like the execution
 * parameters; (0, -1, 0) turns them off.
 *   budget_cycles    limit of every grid-barrier wait of the persistent level
 *                    kernel in clock cycles (0: the default, 2^31, about a second)
 *   skip_block       a block of that kernel that never reaches the launch's first
 *                    barrier (-1: none), so that the other blocks' waits run out
 *   net_stall_polls  > 0: every tensor-core kernel of the proposal net first waits
 *                    that many polls on an mbarrier that nothing completes, then
 *                    reports the timeout, issues no MMA and returns
 * A wait that runs out sets device status code 3 (ff_device_status). */
ff_status ff_set_wait_test(long long budget_cycles, int skip_block, int net_stall_polls);
ff_status ff_get_exec_params(ff_exec_params *e);

/* Learned proposal net (not in the paper). A small convolutional net reads the
 * 1/8-scale images of both frames and emits K flow candidates per point of the
 * coarsest search grid (spacing 8, k = 3); they are passed to ff_flow_fields as
 * `proposals` and tried after the kd-tree candidates under the exact integer
 * data term (strict-less), so they can only replace a kd result with a lower E_d.
 * Layers: four 3x3 convolutions with dilations dil[0..3] and zero padding,
 * channels 6 -> c1 -> c2 -> c3 -> 2K (each <= 64), ReLU between layers, BF16
 * operands and FP32 accumulation on the tensor cores (tcgen05, accumulator in
 * tensor memory). Every wait inside those kernels is bounded; one that runs out
 * sets the device status word at the start of the workspace (ff_device_status). Parameters are one FP32
 * vector, per layer W[cout][cin][3][3] then b[cout]. Tensors are NCHW fp32:
 * x [B][6][Gy][Gx], out [B][2K][Gy][Gx] with Gx = ceil(W/8), Gy = ceil(H/8);
 * out channel 2k (2k+1) is the x (y) flow of candidate k in units of
 * flow_scale pixels. */
typedef struct ff_net_desc {
  int32_t cin, c1, c2, c3, k;
  int32_t dil[4];
} ff_net_desc;
ff_status ff_net_param_count(const ff_net_desc *d, size_t *n);
ff_status ff_net_workspace_size(const ff_net_desc *d, int B, int Gx, int Gy, size_t *bytes);
/* x from B pairs of W x H frames stored back to back ([B][H][W][3] each): the
 * rounded mean of every 8x8 block per channel (as in ff_smooth's area step),
 * scaled to v/255 - 0.5; channels 0-2 frame 1, 3-5 frame 2. */
ff_status ff_net_input(const uint8_t *I1, const uint8_t *I2, int B, int W, int H, float *x,
                       void *stream);
/* Forward pass; keeps the activations in ws for ff_net_backward. */
ff_status ff_net_forward(const ff_net_desc *d, const float *params, const float *x, int B, int Gx,
                         int Gy, float *out, void *ws, size_t ws_bytes, void *stream);
/* Relaxed winner-takes-all L1 loss: for every labelled point (valid != 0) the
 * candidate nearest to the label (L1, first on ties) has weight 1 - alpha, the
 * others alpha / (K - 1); the loss is averaged over labelled points. label:
 * int16 [B][Gy][Gx][2] in pixels. Writes *loss (device float), dout = dloss/dout
 * and *count (device int32, labelled points). */
ff_status ff_net_loss(const ff_net_desc *d, const float *out, const int16_t *label,
                      const uint8_t *valid, int B, int Gx, int Gy, float flow_scale, float alpha,
                      float *loss, float *dout, int32_t *count, void *stream);
/* Backward pass of the last forward (same ws): grads = dloss/dparams. Weight
 * gradients are summed with atomics, so their FP32 rounding order varies. */
ff_status ff_net_backward(const ff_net_desc *d, const float *params, const float *dout, int B,
                          int Gx, int Gy, float *grads, void *ws, size_t ws_bytes, void *stream);
/* Adam (Kingma and Ba, 2015) step `step` (1-based) with bias correction. */
ff_status ff_net_adam(size_t n, float *params, const float *grads, float *m, float *v, int step,
                      float lr, float b1, float b2, float eps, void *stream);
/* Integer proposals rint(out * flow_scale), int16 [B][Gy][Gx][K][2]. */
ff_status ff_net_proposals(const ff_net_desc *d, const float *out, int B, int Gx, int Gy,
                           float flow_scale, int16_t *proposals, void *stream);

/* Device-side status word kept at the start of a workspace: 0 when every
 * device check passed, else the first error code raised with two coordinates
 * saying where: 1 an index out of range that was skipped instead of read (a
 * kd-tree split dimension outside [0, 27) or leaf entry outside [0, W*H) given to
 * ff_kdtree_init: grid point, node or leaf position), 2 an inconsistent kd
 * partition count (node, level), 3 a bounded wait that ran out (block
 * coordinates). Synchronises `stream`, then copies 16 bytes device->host. */
ff_status ff_device_status(const void *ws, uint32_t *code, int32_t *x, int32_t *y, void *stream);

/* Execution counters of the library, for benchmarking (not in the paper).
 * ff_profile_enable(on): bit 0 records CUDA events around every propagation
 * kernel launch (on the stream it was issued on); bit 1 counts the propagation
 * kernels' candidate evaluations on the device; bit 2 records a timing event at
 * every phase boundary of ff_flow_fields / ff_flow_fields_batch on the stream
 * that ran the phase. None is recorded inside ff_graph_create. Host-only calls,
 * not thread-safe against concurrent library calls.
 *   ff_profile_reset     clears the launch counter and the recorded events, and
 *                        (bit 1 set) the evaluation counters (synchronous memset)
 *   ff_profile_read      kernels launched since the reset; summed duration (ms)
 *                        and count of the recorded propagation launches
 *                        (synchronises the recorded events)
 *   ff_profile_levels    the same per level: ms[l], launches[l] for spacing
 *                        n = 2^l, l = 0..4 (5 entries each)
 *   ff_profile_marks     the recorded phase marks in order (at most cap): tags[i]
 *                        = 100 * group + phase, ms[i] = time since the first
 *                        mark; group 0/1/2 = forward / first / second backward
 *                        flow, 3 = shared work; phase 0 start, 1 pyramid done,
 *                        2 features, 3 kd build, 4 kd query, 10 + l level 2^l
 *                        searched, 20 flows joined, 21 filter done; *n = marks
 *                        recorded (synchronises them)
 *   ff_profile_evals     counts[r][l][kind], r = 0..8 (patch radius; 0 unused),
 *                        l = 0..4 (n = 2^l), kinds: 0 incremental with the target
 *                        in the kernel's staged shared-memory window, 1 incremental
 *                        with the target gathered from the census planes, 2 full
 *                        E_d in the window, 3 full E_d gathered (the SIFT flow
 *                        pass kernels gather every target from the colour array:
 *                        kinds 1 and 3); 180 uint64 in total. An incremental evaluation reads 2 (2r+1) target
 *                        taps, a full one (2r+1)^2. Synchronises the device. */
ff_status ff_profile_enable(int on);
ff_status ff_profile_reset(void);
ff_status ff_profile_read(uint64_t *launches, double *prop_ms, uint64_t *prop_launches);
ff_status ff_profile_levels(double *ms, uint64_t *launches);
ff_status ff_profile_marks(int32_t *tags, double *ms, int cap, int *n);
ff_status ff_profile_evals(uint64_t *counts);

/* Measurement probes (not in the paper): the roofline denominators of the search
 * kernels, measured on the running GPU. Each enqueues `blocks` CTAs of 256
 * threads on `stream` and returns at once; the caller times the launch with CUDA
 * events. sink: device uint32 [blocks * 256], overwritten (keeps the work live).
 *   ff_probe_popc       8 independent xor/popcount/add chains per thread on
 *                       registers: 4096 * iters popcounts per CTA
 *   ff_probe_smem_taps  census taps with both words from shared memory,
 *                       conflict-free: 4096 * iters taps per CTA
 *   ff_probe_l2_gather  reads of buf (device, 16-byte aligned, `words` a power
 *                       of two >= 1024; L2-resident when smaller than the L2)
 *                       through ld.global.cg, 8 loads in flight per thread:
 *                       mode 0 a random 4-byte word per lane, mode 1 a random
 *                       16-byte line per lane, mode 2 512 contiguous bytes per
 *                       warp at a random aligned position. *bytes (host, may be
 *                       NULL) = bytes the launch reads. */
ff_status ff_probe_popc(uint32_t *sink, int blocks, int iters, void *stream);
ff_status ff_probe_smem_taps(uint32_t *sink, int blocks, int iters, void *stream);
ff_status ff_probe_l2_gather(const uint32_t *buf, size_t words, int mode, uint32_t *sink,
                             int blocks, int iters, uint64_t *bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FLOWFIELDS_H */
