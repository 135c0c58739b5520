/*
 * Flow Fields CPU oracle (Bailer, Taetz, Stricker, ICCV 2015).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, step-by-step statement
 * of what the GPU library computes. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load it. It shares no code, header, table or
 * generator with the CUDA library: every table it needs it derives itself.
 *
 * Every function names the passage of the paper it follows. Where the paper is
 * silent or garbled the reading taken is stated beside the code.
 *
 * Conventions
 *   images       uint8, H x W x 3 (RGB, or L a b after the colour step), row major
 *   census       uint32 per pixel, H x W
 *   level grids  at spacing n the grid has Gx = ceil(W/n) by Gy = ceil(H/n) points;
 *                grid point (gx, gy) sits on pixel (n*gx, n*gy)
 *   flows        int32 pairs (dx, dy) per grid point, target = pixel + flow
 *   costs        int32 per grid point; COST_UNSET marks a point without a flow
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define COST_UNSET INT32_MAX
#define NFEAT 27

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int imin(int a, int b) { return a < b ? a : b; }

/* floor(a / b) for b > 0 */
static int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) q -= 1;
  return q;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1 / 3.3: the paper computes WHT features and census in CIELab.      */
/* Integer CIELab of an 8-bit sRGB image (reading: D65 white, sRGB primaries   */
/* of IEC 61966-2-1; everything after the 256-entry decoding table is exact   */
/* integer arithmetic, so both implementations can agree bit for bit):         */
/*   1. decode: lin = round(65536 * g(v / 255)), g(c) = c / 12.92 for          */
/*      c <= 0.04045, else ((c + 0.055) / 1.055)^2.4 (1.0 = 65536)             */
/*   2. X/Xn, Y/Yn, Z/Zn: the sRGB->XYZ matrix with each row divided by the     */
/*      white point's component, in Q14, every row rounded so that it sums to  */
/*      exactly 16384 (the residual on its largest entry): a grey pixel gives  */
/*      three equal values. t = (row . lin + 8192) >> 14.                     */
/*   3. f(t) in Q16 (t / 65536 in [0, 1]): the largest y with y^3 <= t * 2^32   */
/*      (= floor(65536 cbrt(t / 65536))) when t / 65536 > (6/29)^3, i.e.       */
/*      t * 29^3 > 6^3 * 65536; else the line t / (3 (6/29)^2) + 4/29, i.e.    */
/*      (29 * 841 * t + 108 * 4 * 65536) / (108 * 29), rounded half up.        */
/*   4. L = 116 f(Y) - 16, a = 500 (f(X) - f(Y)), b = 200 (f(Y) - f(Z));        */
/*      stored as uint8: L * 255 / 100, a + 128, b + 128, each rounded half up */
/*      and clamped to [0, 255].                                              */
/* ------------------------------------------------------------------------ */
static const double SRGB_TO_XYZ[3][3] = {
    {0.4124, 0.3576, 0.1805}, {0.2126, 0.7152, 0.0722}, {0.0193, 0.1192, 0.9505}};

/* Step 1: the decoding table. */
void ffo_lab_gamma_table(int32_t *lin) {
  for (int v = 0; v < 256; v++) {
    double c = v / 255.0;
    double g = c <= 0.04045 ? c / 12.92 : pow((c + 0.055) / 1.055, 2.4);
    lin[v] = (int32_t)floor(g * 65536.0 + 0.5);
  }
}

/* Step 2: the white-normalised matrix rows in Q14, each summing to 16384. */
void ffo_lab_matrix(int32_t *m /* [3][3] */) {
  for (int i = 0; i < 3; i++) {
    double white = SRGB_TO_XYZ[i][0] + SRGB_TO_XYZ[i][1] + SRGB_TO_XYZ[i][2];
    int sum = 0, big = 0;
    for (int j = 0; j < 3; j++) {
      m[3 * i + j] = (int32_t)floor(SRGB_TO_XYZ[i][j] / white * 16384.0 + 0.5);
      sum += m[3 * i + j];
      if (SRGB_TO_XYZ[i][j] > SRGB_TO_XYZ[i][big]) big = j;
    }
    m[3 * i + big] += 16384 - sum;
  }
}

/* Step 3: f(t), t in [0, 65536]. The cube root by bisection on integers. */
int32_t ffo_lab_f(int32_t t) {
  if ((int64_t)t * 24389 > (int64_t)216 * 65536) { /* t/65536 > (6/29)^3 */
    int64_t target = (int64_t)t << 32, lo = 0, hi = 65536; /* hi^3 = 2^48 >= target */
    while (lo < hi) { /* largest y with y^3 <= target */
      int64_t mid = (lo + hi + 1) / 2;
      if (mid * mid * mid <= target) lo = mid;
      else hi = mid - 1;
    }
    return (int32_t)lo;
  }
  return (int32_t)floor_div((int64_t)29 * 841 * t + (int64_t)108 * 4 * 65536 + 1566, 3132);
}

static int lab_round_clamp(int64_t num, int64_t den, int offset) { /* round half up */
  int64_t v = floor_div(2 * num + den, 2 * den) + offset;
  return v < 0 ? 0 : (v > 255 ? 255 : (int)v);
}

/* Steps 1-4 for every pixel: img (RGB) -> out (L, a, b as uint8), H x W x 3. */
void ffo_rgb_to_lab(const uint8_t *img, int W, int H, uint8_t *out) {
  int32_t lin[256], m[9];
  ffo_lab_gamma_table(lin);
  ffo_lab_matrix(m);
  for (size_t p = 0; p < (size_t)W * H; p++) {
    int64_t c[3] = {lin[img[3 * p]], lin[img[3 * p + 1]], lin[img[3 * p + 2]]};
    int32_t f[3];
    for (int i = 0; i < 3; i++) {
      int64_t t = (m[3 * i] * c[0] + m[3 * i + 1] * c[1] + m[3 * i + 2] * c[2] + 8192) >> 14;
      f[i] = ffo_lab_f((int32_t)t);
    }
    out[3 * p] = (uint8_t)lab_round_clamp(((int64_t)116 * f[1] - 16 * 65536) * 255, 100 * 65536, 0);
    out[3 * p + 1] = (uint8_t)lab_round_clamp((int64_t)500 * (f[0] - f[1]), 65536, 128);
    out[3 * p + 2] = (uint8_t)lab_round_clamp((int64_t)200 * (f[1] - f[2]), 65536, 128);
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: the smoothed full-resolution image I^n. Area downsampling by n,  */
/* then Lanczos upsampling back to full resolution.                          */
/* ------------------------------------------------------------------------ */

/* Area downsampling: the mean over the in-image part of each n x n block,
 * rounded half up in integer arithmetic: (sum + cnt/2) / cnt. */
void ffo_area_down(const uint8_t *img, int W, int H, int n, uint8_t *out) {
  int Wc = (W + n - 1) / n, Hc = (H + n - 1) / n;
  for (int j = 0; j < Hc; j++)
    for (int i = 0; i < Wc; i++)
      for (int c = 0; c < 3; c++) {
        int sum = 0, cnt = 0;
        for (int y = j * n; y < imin(j * n + n, H); y++)
          for (int x = i * n; x < imin(i * n + n, W); x++) {
            sum += img[((size_t)y * W + x) * 3 + c];
            cnt++;
          }
        out[((size_t)j * Wc + i) * 3 + c] = (uint8_t)((sum + cnt / 2) / cnt);
      }
}

/* Lanczos kernel with a = 3 (the paper does not give the order). */
static double lanczos3(double t) {
  if (t == 0.0) return 1.0;
  if (fabs(t) >= 3.0) return 0.0;
  double pt = M_PI * t;
  return 3.0 * sin(pt) * sin(pt / 3.0) / (pt * pt);
}

/* Per-phase Lanczos taps for integer upsampling by n.
 * Coarse sample j is centred on full-resolution position j*n + (n-1)/2, so the
 * full-resolution pixel x sits at coarse coordinate u = (2x - n + 1) / (2n).
 * With j0 = floor(u) and f = u - j0 the six taps are j0-2 .. j0+3 with weight
 * L(f - k). The weights are normalised to sum 1, scaled to Q14 and rounded half
 * away from zero; the tap of largest magnitude (first on ties) takes the
 * residual so that each phase sums to exactly 16384.
 * Outputs: base[phi] = j0 for x = phi (x = q*n + phi has base q + base[phi]),
 *          w[phi*6 + (k+2)]. */
void ffo_lanczos_table(int n, int32_t *base, int32_t *w) {
  for (int phi = 0; phi < n; phi++) {
    int64_t num = 2 * phi - n + 1, den = 2 * (int64_t)n;
    int64_t j0 = floor_div(num, den);
    double f = (double)(num - den * j0) / (double)den;
    double wd[6], s = 0.0;
    for (int k = -2; k <= 3; k++) {
      wd[k + 2] = lanczos3(f - k);
      s += wd[k + 2];
    }
    int32_t tot = 0;
    int big = 0;
    for (int t = 0; t < 6; t++) {
      double v = 16384.0 * wd[t] / s;
      int32_t q = (int32_t)(v >= 0 ? floor(v + 0.5) : -floor(-v + 0.5));
      w[phi * 6 + t] = q;
      tot += q;
    }
    for (int t = 1; t < 6; t++)
      if (abs(w[phi * 6 + t]) > abs(w[phi * 6 + big])) big = t;
    w[phi * 6 + big] += 16384 - tot;
    base[phi] = (int32_t)j0;
  }
}

/* I^n from I: area down by n, then separable Lanczos-3 up to W x H.
 * Horizontal pass keeps an unrounded int32 Q14 value per coarse row; the vertical
 * pass accumulates in int64 and rounds (acc + 2^27) >> 28, clamped to [0, 255].
 * For n = 1 the image is copied. */
void ffo_smooth(const uint8_t *img, int W, int H, int n, uint8_t *out) {
  if (n == 1) {
    memcpy(out, img, (size_t)W * H * 3);
    return;
  }
  int Wc = (W + n - 1) / n, Hc = (H + n - 1) / n;
  uint8_t *D = malloc((size_t)Wc * Hc * 3);
  int32_t *hz = malloc(sizeof(int32_t) * (size_t)Hc * W * 3);
  int32_t *base = malloc(sizeof(int32_t) * n), *wt = malloc(sizeof(int32_t) * 6 * n);
  ffo_area_down(img, W, H, n, D);
  ffo_lanczos_table(n, base, wt);
  for (int yc = 0; yc < Hc; yc++)
    for (int x = 0; x < W; x++) {
      int phi = x % n, j0 = x / n + base[phi];
      for (int c = 0; c < 3; c++) {
        int32_t acc = 0;
        for (int k = -2; k <= 3; k++) {
          int j = clampi(j0 + k, 0, Wc - 1);
          acc += wt[phi * 6 + k + 2] * (int32_t)D[((size_t)yc * Wc + j) * 3 + c];
        }
        hz[((size_t)yc * W + x) * 3 + c] = acc;
      }
    }
  for (int y = 0; y < H; y++) {
    int phi = y % n, j0 = y / n + base[phi];
    for (int x = 0; x < W; x++)
      for (int c = 0; c < 3; c++) {
        int64_t acc = 0;
        for (int k = -2; k <= 3; k++) {
          int j = clampi(j0 + k, 0, Hc - 1);
          acc += (int64_t)wt[phi * 6 + k + 2] * hz[((size_t)j * W + x) * 3 + c];
        }
        int64_t v = floor_div(acc + ((int64_t)1 << 27), (int64_t)1 << 28);
        out[((size_t)y * W + x) * 3 + c] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
      }
  }
  free(D);
  free(hz);
  free(base);
  free(wt);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3: census transform data term.                                     */
/* Reading: 3x3 census per colour channel on I^n with neighbour spacing n.   */
/* Bit (8c + o) is set when channel c of neighbour o is darker than the      */
/* centre; the 8 neighbours are taken in raster order skipping the centre;  */
/* coordinates are clamped into the image.                                   */
/* ------------------------------------------------------------------------ */
void ffo_census(const uint8_t *imgn, int W, int H, int n, uint32_t *out) {
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      uint32_t code = 0;
      for (int c = 0; c < 3; c++) {
        int centre = imgn[((size_t)y * W + x) * 3 + c];
        int o = 0;
        for (int dy = -1; dy <= 1; dy++)
          for (int dx = -1; dx <= 1; dx++) {
            if (dx == 0 && dy == 0) continue;
            int xx = clampi(x + n * dx, 0, W - 1), yy = clampi(y + n * dy, 0, H - 1);
            if (imgn[((size_t)yy * W + xx) * 3 + c] < centre) code |= 1u << (8 * c + o);
            o++;
          }
      }
      out[(size_t)y * W + x] = code;
    }
}

/* Sec. 3.1: the random search's subpixel targets take their colours from
 * bilinear interpolation. Reading (subpel q in {1, 2, 4}): flows are kept in
 * units of 1/q pixel; a target X = q x + a, Y = q y + b (0 <= a, b < q) reads
 * the census of the image interpolated at (x + a/q, y + b/q):
 *   J(x, y) = sum_{i,j in {0,1}} wx_i wy_j I^n(clamp(x + i), clamp(y + j)),
 *   wx_0 = q - a, wx_1 = a, wy_0 = q - b, wy_1 = b
 * (q^2 times the interpolated colour, kept exact), with the census of J at
 * spacing n as in ffo_census. Phase (0, 0) is q^2 I^n: the plain census. */
void ffo_census_subpel(const uint8_t *imgn, int W, int H, int n, int q, int a, int b,
                       uint32_t *out) {
  size_t N = (size_t)W * H;
  int32_t *J = malloc(sizeof(int32_t) * N * 3);
  int wx[2] = {q - a, a}, wy[2] = {q - b, b};
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++)
      for (int c = 0; c < 3; c++) {
        int32_t v = 0;
        for (int j = 0; j < 2; j++)
          for (int i = 0; i < 2; i++)
            v += wx[i] * wy[j] *
                 imgn[((size_t)clampi(y + j, 0, H - 1) * W + clampi(x + i, 0, W - 1)) * 3 + c];
        J[((size_t)y * W + x) * 3 + c] = v;
      }
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      uint32_t code = 0;
      for (int c = 0; c < 3; c++) {
        int32_t centre = J[((size_t)y * W + x) * 3 + c];
        int o = 0;
        for (int dy = -1; dy <= 1; dy++)
          for (int dx = -1; dx <= 1; dx++) {
            if (dx == 0 && dy == 0) continue;
            int xx = clampi(x + n * dx, 0, W - 1), yy = clampi(y + n * dy, 0, H - 1);
            if (J[((size_t)yy * W + xx) * 3 + c] < centre) code |= 1u << (8 * c + o);
            o++;
          }
      }
      out[(size_t)y * W + x] = code;
    }
  free(J);
}

static int popcount32(uint32_t v) { return __builtin_popcount(v); }

/* E_d of Eq. 1/3/4 with the census data term: the summed census Hamming
 * distance over the (2r+1)^2 taps of the subsampled patches P^n_r (Eq. 3),
 * each tap clamped into the image. */
int32_t ffo_patch_cost(const uint32_t *Cs, const uint32_t *Ct, int W, int H, int n, int r,
                       int x1, int y1, int x2, int y2) {
  int32_t e = 0;
  for (int v = -r; v <= r; v++)
    for (int u = -r; u <= r; u++) {
      int xs = clampi(x1 + n * u, 0, W - 1), ys = clampi(y1 + n * v, 0, H - 1);
      int xt = clampi(x2 + n * u, 0, W - 1), yt = clampi(y2 + n * v, 0, H - 1);
      e += popcount32(Cs[(size_t)ys * W + xs] ^ Ct[(size_t)yt * W + xt]);
    }
  return e;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3, the second data term: SIFT flow. Every pixel gets a 128-D SIFT  */
/* vector, reduced by PCA to S dimensions ("SIFT flow colours"); E_d is the  */
/* L2 distance between colours, summed over the patch taps. The paper names  */
/* the descriptor only; readings (all integer, so both sides agree exactly): */
/*   grey      g = R + G + B of the input frame (0..765)                       */
/*   gradient  gx = g(x+1, y) - g(x-1, y), gy = g(x, y+1) - g(x, y-1),         */
/*             coordinates clamped                                           */
/*   8 orientations: the half-wave rectified derivative along direction k*45  */
/*             degrees (x right, y down): o_k = max(0, gx C_k + gy S_k), with */
/*             (C_k, S_k) = 256 (cos, sin) rounded, 1/sqrt 2 -> 181/256       */
/*   4 x 4 cells of SIFT_CELL x SIFT_CELL pixels: cell (i, j) of pixel p sums */
/*             o_k over x in [px + (i-2) c, px + (i-1) c), y likewise with j, */
/*             coordinates clamped (flat spatial weights)                     */
/*   element   d = (4 j + i) * 8 + k                                          */
/*   normalise Lowe's unit length, clip at 0.2, unit length again, x 512,     */
/*             clamp 255, in integers: N2 = sum h^2, t = isqrt(N2 / 25),      */
/*             h' = min(h, t), M2 = sum h'^2, q = min(255, isqrt(2^18 h'^2 /  */
/*             M2)) (integer divisions); M2 = 0 gives q = 0                   */
/* ------------------------------------------------------------------------ */
#define SIFT_CELL 3
#define SIFT_DIM 128

static const int SIFT_C[8] = {256, 181, 0, -181, -256, -181, 0, 181};
static const int SIFT_S[8] = {0, 181, 256, 181, 0, -181, -256, -181};

/* floor(sqrt(x)) by bisection on the integers */
static uint64_t isqrt_u64(uint64_t x) {
  uint64_t lo = 0, hi = 1ull << 32; /* hi^2 > x for every x < 2^64 */
  while (hi - lo > 1) {
    uint64_t mid = lo + (hi - lo) / 2;
    if ((unsigned __int128)mid * mid <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

uint64_t ffo_isqrt(uint64_t x) { return isqrt_u64(x); }

static int grey_at(const uint8_t *img, int W, int H, int x, int y) {
  const uint8_t *p = img + 3 * ((size_t)clampi(y, 0, H - 1) * W + clampi(x, 0, W - 1));
  return p[0] + p[1] + p[2];
}

/* The 8 orientation responses at every pixel: o[(y W + x) 8 + k]. */
void ffo_sift_orient(const uint8_t *img, int W, int H, int32_t *o) {
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      int gx = grey_at(img, W, H, x + 1, y) - grey_at(img, W, H, x - 1, y);
      int gy = grey_at(img, W, H, x, y + 1) - grey_at(img, W, H, x, y - 1);
      for (int k = 0; k < 8; k++) {
        int v = gx * SIFT_C[k] + gy * SIFT_S[k];
        o[((size_t)y * W + x) * 8 + k] = v > 0 ? v : 0;
      }
    }
}

/* Dense SIFT: desc[(y W + x) 128 + d], uint8. */
void ffo_sift_descriptors(const uint8_t *img, int W, int H, uint8_t *desc) {
  size_t N = (size_t)W * H;
  int32_t *o = malloc(sizeof(int32_t) * 8 * N);
  ffo_sift_orient(img, W, H, o);
  int64_t h[SIFT_DIM];
  for (int py = 0; py < H; py++)
    for (int px = 0; px < W; px++) {
      for (int j = 0; j < 4; j++)
        for (int i = 0; i < 4; i++)
          for (int k = 0; k < 8; k++) {
            int64_t acc = 0;
            for (int v = (j - 2) * SIFT_CELL; v < (j - 1) * SIFT_CELL; v++)
              for (int u = (i - 2) * SIFT_CELL; u < (i - 1) * SIFT_CELL; u++) {
                int x = clampi(px + u, 0, W - 1), y = clampi(py + v, 0, H - 1);
                acc += o[((size_t)y * W + x) * 8 + k];
              }
            h[(4 * j + i) * 8 + k] = acc;
          }
      uint64_t N2 = 0;
      for (int d = 0; d < SIFT_DIM; d++) N2 += (uint64_t)(h[d] * h[d]);
      uint64_t t = isqrt_u64(N2 / 25);
      uint64_t M2 = 0;
      for (int d = 0; d < SIFT_DIM; d++) {
        if ((uint64_t)h[d] > t) h[d] = (int64_t)t;
        M2 += (uint64_t)(h[d] * h[d]);
      }
      uint8_t *out = desc + ((size_t)py * W + px) * SIFT_DIM;
      for (int d = 0; d < SIFT_DIM; d++) {
        uint64_t qv = 0;
        if (M2 > 0) qv = isqrt_u64(((uint64_t)(h[d] * h[d]) << 18) / M2);
        out[d] = (uint8_t)(qv > 255 ? 255 : qv);
      }
    }
  free(o);
}

/* PCA statistics of N descriptors, added to the outputs: sum[i] += sum of q_i,
 * gram[i 128 + j] += sum of q_i q_j (exact). */
void ffo_sift_moments(const uint8_t *desc, int N, uint64_t *sum, uint64_t *gram) {
  for (int p = 0; p < N; p++) {
    const uint8_t *q = desc + (size_t)p * SIFT_DIM;
    for (int i = 0; i < SIFT_DIM; i++) {
      sum[i] += q[i];
      for (int j = 0; j < SIFT_DIM; j++) gram[i * SIFT_DIM + j] += (uint64_t)q[i] * q[j];
    }
  }
}

/* Centring offsets of a quantised basis B[S][128] (components in units of
 * 2^-12): o_s = 2^11 - round(sum_i B_si mean_i), the rounding half up, exact
 * from the integer sums of `count` descriptors. */
void ffo_sift_pca_offset(const int16_t *B, int S, const uint64_t *sum, int64_t count,
                         int32_t *off) {
  for (int s = 0; s < S; s++) {
    int64_t num = 0;
    for (int i = 0; i < SIFT_DIM; i++) num += (int64_t)B[s * SIFT_DIM + i] * (int64_t)sum[i];
    off[s] = (int32_t)(2048 - floor_div(2 * num + count, 2 * count));
  }
}

/* SIFT flow colours: channel s of pixel p is clamp(128 + floor((sum_i B_si q_i
 * + o_s) / 2^12), 0, 255). Stored in S/3 groups of three channels, each group an
 * H x W x 3 image (so that each group smooths like a colour image, Sec. 3.2):
 * col[(s/3) N 3 + p 3 + s%3]. */
void ffo_sift_colors(const uint8_t *desc, int W, int H, const int16_t *B, const int32_t *off,
                     int S, uint8_t *col) {
  size_t N = (size_t)W * H;
  for (size_t p = 0; p < N; p++) {
    const uint8_t *q = desc + p * SIFT_DIM;
    for (int s = 0; s < S; s++) {
      int64_t acc = off[s];
      for (int i = 0; i < SIFT_DIM; i++) acc += (int64_t)B[s * SIFT_DIM + i] * q[i];
      int64_t v = 128 + floor_div(acc, 4096);
      col[(size_t)(s / 3) * N * 3 + p * 3 + s % 3] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
    }
  }
}

/* Distance of two SIFT flow colours: the Euclidean norm in fixed point with 4
 * fractional bits, floor(16 sqrt(sum (a_s - b_s)^2)). */
int32_t ffo_sift_tap(const uint8_t *Ks, const uint8_t *Kt, int S, size_t N, size_t ps,
                     size_t pt) {
  uint64_t acc = 0;
  for (int s = 0; s < S; s++) {
    size_t g = (size_t)(s / 3) * N * 3;
    int d = (int)Ks[g + ps * 3 + s % 3] - (int)Kt[g + pt * 3 + s % 3];
    acc += (uint64_t)(d * d);
  }
  return (int32_t)isqrt_u64(acc * 256);
}

/* E_d with the SIFT flow data term: the tap distances over the (2r+1)^2 taps of
 * P^n_r (Eq. 3) of the level-n colours, each tap clamped into the image. */
int32_t ffo_sift_patch_cost(const uint8_t *Ks, const uint8_t *Kt, int S, int W, int H, int n,
                            int r, int x1, int y1, int x2, int y2) {
  int32_t e = 0;
  size_t N = (size_t)W * H;
  for (int v = -r; v <= r; v++)
    for (int u = -r; u <= r; u++) {
      int xs = clampi(x1 + n * u, 0, W - 1), ys = clampi(y1 + n * v, 0, H - 1);
      int xt = clampi(x2 + n * u, 0, W - 1), yt = clampi(y2 + n * v, 0, H - 1);
      e += ffo_sift_tap(Ks, Kt, S, N, (size_t)ys * W + xs, (size_t)yt * W + xt);
    }
  return e;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: Walsh-Hadamard patch features.                                 */
/* Reading: the window of L = 2r+1 pixels is split into halves floor(L/2),  */
/* ceil(L/2) (the paper's uneven r / r+1 split), and each half the same way,*/
/* giving 4 blocks. The 1-D Walsh functions in sequency order over the 4    */
/* blocks are (++++), (++--), (+--+), (+-+-). The 9 features per channel    */
/* are rows-function i times columns-function j, i, j in {0, 1, 2}; feature */
/* index 9c + 3i + j; pixels are read with clamped coordinates.             */
/* ------------------------------------------------------------------------ */
void ffo_wht_blocks(int L, int32_t *size4) {
  int h0 = L / 2, h1 = L - h0;
  size4[0] = h0 / 2;
  size4[1] = h0 - h0 / 2;
  size4[2] = h1 / 2;
  size4[3] = h1 - h1 / 2;
}

/* nb (<= 4) 1-D Walsh functions over L pixels, out[i*L + t] in {-1, +1}. */
void ffo_wht_basis_1d(int L, int nb, int32_t *out) {
  static const int sgn[4][4] = {{1, 1, 1, 1}, {1, 1, -1, -1}, {1, -1, -1, 1}, {1, -1, 1, -1}};
  int32_t sz[4];
  ffo_wht_blocks(L, sz);
  for (int i = 0; i < nb; i++) {
    int t = 0;
    for (int b = 0; b < 4; b++)
      for (int k = 0; k < sz[b]; k++) out[i * L + t++] = sgn[i][b];
  }
}

/* General form: window of L pixels starting at x - (L-1)/2 (centred for odd L),
 * nb x nb bases per channel, out[k*3*nb*nb + c*nb*nb + i*nb + j]. The odd-L,
 * nb = 3 case is the feature vector; L = 4 with nb = 4 is the complete
 * Walsh-Hadamard transform of a 4x4 patch. */
void ffo_wht_features_general(const uint8_t *img, int W, int H, int L, int nb,
                              const int32_t *pts, int npts, int32_t *out) {
  int h = (L - 1) / 2, nf = 3 * nb * nb;
  int32_t *w = malloc(sizeof(int32_t) * nb * L);
  int64_t *rowsum = malloc(sizeof(int64_t) * L * 3 * nb);
  ffo_wht_basis_1d(L, nb, w);
  int total = pts ? npts : W * H;
  for (int k = 0; k < total; k++) {
    int x = pts ? pts[2 * k] : k % W, y = pts ? pts[2 * k + 1] : k / W;
    /* rowsum[v][c][j] = sum_u w_j(u) I_c(x - h + u, y - h + v) */
    for (int v = 0; v < L; v++) {
      int yy = clampi(y - h + v, 0, H - 1);
      for (int c = 0; c < 3; c++)
        for (int j = 0; j < nb; j++) {
          int64_t s = 0;
          for (int u = 0; u < L; u++) {
            int xx = clampi(x - h + u, 0, W - 1);
            s += (int64_t)w[j * L + u] * img[((size_t)yy * W + xx) * 3 + c];
          }
          rowsum[(v * 3 + c) * nb + j] = s;
        }
    }
    for (int c = 0; c < 3; c++)
      for (int i = 0; i < nb; i++)
        for (int j = 0; j < nb; j++) {
          int64_t s = 0;
          for (int v = 0; v < L; v++) s += (int64_t)w[i * L + v] * rowsum[(v * 3 + c) * nb + j];
          out[(size_t)k * nf + c * nb * nb + i * nb + j] = (int32_t)s;
        }
  }
  free(w);
  free(rowsum);
}

/* Features at the listed pixels (pts = NULL: every pixel in raster order).
 * The patch P_r is the non-subsampled one (Sec. 3.2: WHTs use P_r even in the
 * hierarchical search). out[k*27 + 9c + 3i + j]. */
void ffo_wht_features(const uint8_t *img, int W, int H, int r, const int32_t *pts, int npts,
                      int32_t *out) {
  ffo_wht_features_general(img, W, H, 2 * r + 1, 3, pts, npts, out);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: kd-tree over the 27-D vectors of all target pixels, leaf size l, */
/* split in the dimension of maximal spread at the median.                   */
/* Reading: a perfect tree of depth D = smallest d with ceil(N / 2^d) <= l.  */
/* Spread = max - min (lowest dimension on ties). A node of m points sends   */
/* the first floor(m/2) under the order (value, pixel index) to the left;   */
/* the split value is the value of the first point on the right. Nodes are  */
/* in heap order (children of i are 2i+1, 2i+2).                            */
/* ------------------------------------------------------------------------ */
int ffo_kd_depth(int N, int leaf) {
  int d = 0;
  while (((int64_t)N + ((int64_t)1 << d) - 1) / ((int64_t)1 << d) > leaf) d++;
  return d;
}

typedef struct {
  int32_t value, idx;
} kd_key;

static int key_cmp(const void *a, const void *b) {
  const kd_key *x = a, *y = b;
  if (x->value != y->value) return x->value < y->value ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static void kd_node(const int32_t *feat, int32_t *perm, kd_key *tmp, int begin, int end, int depth,
                    int D, int node, int32_t *split_dim, int32_t *split_val) {
  if (depth == D) return;
  int m = end - begin, best = 0;
  int64_t best_spread = -1;
  for (int d = 0; d < NFEAT; d++) {
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    for (int k = begin; k < end; k++) {
      int32_t v = feat[(size_t)perm[k] * NFEAT + d];
      if (v < lo) lo = v;
      if (v > hi) hi = v;
    }
    if ((int64_t)hi - lo > best_spread) {
      best_spread = (int64_t)hi - lo;
      best = d;
    }
  }
  for (int k = 0; k < m; k++) {
    tmp[k].value = feat[(size_t)perm[begin + k] * NFEAT + best];
    tmp[k].idx = perm[begin + k];
  }
  qsort(tmp, m, sizeof(kd_key), key_cmp);
  for (int k = 0; k < m; k++) perm[begin + k] = tmp[k].idx;
  int half = m / 2;
  split_dim[node] = best;
  split_val[node] = tmp[half].value;
  kd_node(feat, perm, tmp, begin, begin + half, depth + 1, D, 2 * node + 1, split_dim, split_val);
  kd_node(feat, perm, tmp, begin + half, end, depth + 1, D, 2 * node + 2, split_dim, split_val);
}

/* perm[N]: pixel indices grouped by leaf (leaf order = heap order of depth D);
 * split_dim / split_val: 2^D - 1 internal nodes. Returns D. */
int ffo_kd_build(const int32_t *feat, int N, int leaf, int32_t *perm, int32_t *split_dim,
                 int32_t *split_val) {
  int D = ffo_kd_depth(N, leaf);
  kd_key *tmp = malloc(sizeof(kd_key) * (size_t)(N > 0 ? N : 1));
  for (int k = 0; k < N; k++) perm[k] = k;
  kd_node(feat, perm, tmp, 0, N, 0, D, 0, split_dim, split_val);
  free(tmp);
  return D;
}

/* Range of leaf `leaf` in perm: halve [0, N) D times along the leaf's path. */
void ffo_kd_leaf_range(int N, int D, int leaf, int32_t *begin, int32_t *end) {
  int b = 0, e = N;
  for (int d = D - 1; d >= 0; d--) {
    int half = (e - b) / 2;
    if ((leaf >> d) & 1) b = b + half;
    else e = b + half;
  }
  *begin = b;
  *end = e;
}

/* Bounded-leaf query without backtracking: at each node go left iff the query
 * value is below the split value. Returns the leaf index in [0, 2^D). */
int ffo_kd_query(const int32_t *split_dim, const int32_t *split_val, int D, const int32_t *q) {
  int node = 0;
  for (int d = 0; d < D; d++)
    node = (q[split_dim[node]] < split_val[node]) ? 2 * node + 1 : 2 * node + 2;
  return node - ((1 << D) - 1);
}

/* ------------------------------------------------------------------------ */
/* Candidates. Reading: a candidate flow f at pixel p is applied with its     */
/* target clamped into the image, f := clamp(p + f) - p, so every flow stays */
/* valid. Replacement needs a strictly lower cost ("if the matching error   */
/* decreases", Sec. 3.1); earlier candidates win ties.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  const uint32_t *Cs;
  const uint32_t *const *Ct; /* target census per subpixel phase b * q + a */
  int W, H, n, r, q;
  int64_t evals;
  /* S > 0: the SIFT flow data term on the level-n colours Ks, Kt (q = 1) */
  const uint8_t *Ks, *Kt;
  int S;
} level_ctx;

/* Flows are in units of 1/q pixel (q = 1: pixels). The target X = q px + fx is
 * clamped to [0, q (W - 1)] (and Y likewise), so it stays inside the image. */
static void try_candidate(level_ctx *L, int px, int py, int fx, int fy, int32_t *flow,
                          int32_t *cost) {
  int q = L->q;
  int X = clampi(q * px + fx, 0, q * (L->W - 1)), Y = clampi(q * py + fy, 0, q * (L->H - 1));
  int32_t e;
  if (L->S > 0) {
    e = ffo_sift_patch_cost(L->Ks, L->Kt, L->S, L->W, L->H, L->n, L->r, px, py, X, Y);
  } else {
    const uint32_t *Ct = L->Ct[(Y % q) * q + X % q];
    e = ffo_patch_cost(L->Cs, Ct, L->W, L->H, L->n, L->r, px, py, X / q, Y / q);
  }
  L->evals++;
  if (e < *cost) {
    *cost = e;
    flow[0] = X - q * px;
    flow[1] = Y - q * py;
  }
}

/* Eq. 1 / Eq. 4: initial flow at the grid points of spacing n from the kd
 * leaf of each point's WHT vector (features of the source image at that
 * point, radius r), reranked by E_d on P^n_r. Leaf entries are scanned in
 * ascending pixel index. Optional proposals (K per grid point, int32 pairs)
 * are tried afterwards in index order under the same strict-less rule.
 * tgt_feat: features of every target pixel; the tree is built here. */
static int64_t kd_init_q(const int32_t *tgt_feat, const uint8_t *src_img, int W, int H, int r,
                         int leaf, const uint32_t *Cs, const uint32_t *const *Ct, int q, int n,
                         const int32_t *proposals, int K, int32_t *flow, int32_t *cost,
                         const uint8_t *Ks, const uint8_t *Kt, int S);

int64_t ffo_kd_init(const int32_t *tgt_feat, const uint8_t *src_img, int W, int H, int r,
                    int leaf, const uint32_t *Cs, const uint32_t *Ct, int n,
                    const int32_t *proposals, int K, int32_t *flow, int32_t *cost) {
  const uint32_t *Ct1[1] = {Ct};
  return kd_init_q(tgt_feat, src_img, W, H, r, leaf, Cs, Ct1, 1, n, proposals, K, flow, cost,
                   NULL, NULL, 0);
}

/* With subpel q the leaf pixels and the proposals (in pixels) become flows of
 * q (x2 - px) in 1/q pixel units. */
static int64_t kd_init_q(const int32_t *tgt_feat, const uint8_t *src_img, int W, int H, int r,
                         int leaf, const uint32_t *Cs, const uint32_t *const *Ct, int q, int n,
                         const int32_t *proposals, int K, int32_t *flow, int32_t *cost,
                         const uint8_t *Ks, const uint8_t *Kt, int S) {
  int N = W * H, Gx = (W + n - 1) / n, Gy = (H + n - 1) / n, G = Gx * Gy;
  int D = ffo_kd_depth(N, leaf);
  int32_t *perm = malloc(sizeof(int32_t) * N);
  int32_t *sd = malloc(sizeof(int32_t) * ((1 << D) + 1));
  int32_t *sv = malloc(sizeof(int32_t) * ((1 << D) + 1));
  int32_t *pts = malloc(sizeof(int32_t) * 2 * G), *qf = malloc(sizeof(int32_t) * NFEAT * G);
  int32_t *cand = malloc(sizeof(int32_t) * (leaf + 1));
  ffo_kd_build(tgt_feat, N, leaf, perm, sd, sv);
  for (int g = 0; g < G; g++) {
    pts[2 * g] = (g % Gx) * n;
    pts[2 * g + 1] = (g / Gx) * n;
  }
  ffo_wht_features(src_img, W, H, r, pts, G, qf);
  level_ctx L = {Cs, Ct, W, H, n, r, q, 0, Ks, Kt, S};
  for (int g = 0; g < G; g++) {
    int px = pts[2 * g], py = pts[2 * g + 1];
    int lf = ffo_kd_query(sd, sv, D, qf + (size_t)g * NFEAT);
    int32_t b, e;
    ffo_kd_leaf_range(N, D, lf, &b, &e);
    int m = e - b;
    for (int k = 0; k < m; k++) cand[k] = perm[b + k];
    /* ascending pixel index */
    for (int i = 1; i < m; i++)
      for (int j = i; j > 0 && cand[j - 1] > cand[j]; j--) {
        int32_t t = cand[j];
        cand[j] = cand[j - 1];
        cand[j - 1] = t;
      }
    int32_t *f = flow + 2 * (size_t)g;
    cost[g] = COST_UNSET;
    f[0] = f[1] = 0;
    for (int k = 0; k < m; k++)
      try_candidate(&L, px, py, q * (cand[k] % W - px), q * (cand[k] / W - py), f, &cost[g]);
    for (int k = 0; k < K; k++)
      try_candidate(&L, px, py, q * proposals[((size_t)g * K + k) * 2],
                    q * proposals[((size_t)g * K + k) * 2 + 1], f, &cost[g]);
  }
  free(perm);
  free(sd);
  free(sv);
  free(pts);
  free(qf);
  free(cand);
  return L.evals;
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers for the random search (Sec. 3.1).            */
/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): add the golden gamma, then   */
/* the 64-bit finaliser. The key packs gx (bits 0-23), gy (24-47), the      */
/* random-search step (48-49), log2 n (50-52) and the flow id (53-54), xored  */
/* into the seed. Lemire's multiply-shift maps each 32-bit half to           */
/* [0, 2R_n]; the low half gives dx, the high half dy.                       */
/* ------------------------------------------------------------------------ */
uint64_t ffo_splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

void ffo_rs_offset(uint64_t seed, int flow_id, int level, int step, int gx, int gy, int Rn,
                   int32_t *d) {
  uint64_t key = seed ^ ((uint64_t)gx & 0xffffff) ^ (((uint64_t)gy & 0xffffff) << 24) ^
                 ((uint64_t)(step & 3) << 48) ^ ((uint64_t)(level & 7) << 50) ^
                 ((uint64_t)(flow_id & 3) << 53);
  uint64_t z = ffo_splitmix64(key);
  uint64_t span = 2 * (uint64_t)Rn + 1;
  d[0] = (int32_t)((((z & 0xffffffffULL) * span) >> 32)) - Rn;
  d[1] = (int32_t)((((z >> 32) * span) >> 32)) - Rn;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1/3.2: propagation (Eq. 2) and random search on the grid of        */
/* spacing n.                                                                 */
/* Reading of Fig. 3c (missing from the text): pass 0 takes its sources from */
/* (x-n, y), (x, y-n) and scans top-down, left to right; pass 1 from (x+n, y),*/
/* (x, y+n), bottom-up, right to left; pass 2 from (x+n, y), (x, y-n),       */
/* top-down, right to left; pass 3 from (x-n, y), (x, y+n), bottom-up, left  */
/* to right. Candidates in order: current, horizontal source, vertical      */
/* source. A source without a flow (COST_UNSET) or outside the grid is       */
/* skipped.                                                                   */
/*                                                                            */
/* Schedules. tile == 0 is the paper's sequential scan over the whole grid.  */
/* tile == T > 0 splits the grid into T x T tiles, with the tile origin      */
/* shifted by T/2 on both axes in odd passes; inside a tile the pass is the  */
/* sequential scan, and a source outside the tile is read from the state at  */
/* the start of the pass.                                                    */
/* ------------------------------------------------------------------------ */
static const int PASS_SRC[4][2][2] = {
    {{-1, 0}, {0, -1}}, {{1, 0}, {0, 1}}, {{1, 0}, {0, -1}}, {{-1, 0}, {0, 1}}};

static void prop_pass(level_ctx *L, int s, int tile, int32_t *flow, int32_t *cost) {
  int n = L->n, Gx = (L->W + n - 1) / n, Gy = (L->H + n - 1) / n, G = Gx * Gy;
  int32_t *snap_f = malloc(sizeof(int32_t) * 2 * G), *snap_c = malloc(sizeof(int32_t) * G);
  memcpy(snap_f, flow, sizeof(int32_t) * 2 * G);
  memcpy(snap_c, cost, sizeof(int32_t) * G);
  int T = tile, off = 0, ntx = 1, nty = 1;
  if (T > 0) {
    off = (s % 2) * (T / 2);
    ntx = (Gx + off + T - 1) / T;
    nty = (Gy + off + T - 1) / T;
  }
  int sx = PASS_SRC[s][0][0], sy = PASS_SRC[s][1][1]; /* scan direction = -source direction */
  for (int ty = 0; ty < nty; ty++)
    for (int tx = 0; tx < ntx; tx++) {
      int x0 = 0, x1 = Gx, y0 = 0, y1 = Gy;
      if (T > 0) {
        x0 = tx * T - off;
        x1 = x0 + T;
        y0 = ty * T - off;
        y1 = y0 + T;
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > Gx) x1 = Gx;
        if (y1 > Gy) y1 = Gy;
      }
      for (int iy = 0; iy < y1 - y0; iy++) {
        int gy = (sy < 0) ? y0 + iy : y1 - 1 - iy;
        for (int ix = 0; ix < x1 - x0; ix++) {
          int gx = (sx < 0) ? x0 + ix : x1 - 1 - ix;
          int g = gy * Gx + gx;
          for (int c = 0; c < 2; c++) {
            int qx = gx + PASS_SRC[s][c][0], qy = gy + PASS_SRC[s][c][1];
            if (qx < 0 || qx >= Gx || qy < 0 || qy >= Gy) continue;
            int q = qy * Gx + qx;
            int in_tile = qx >= x0 && qx < x1 && qy >= y0 && qy < y1;
            const int32_t *fq = in_tile ? flow + 2 * (size_t)q : snap_f + 2 * (size_t)q;
            int32_t cq = in_tile ? cost[q] : snap_c[q];
            if (cq == COST_UNSET) continue;
            try_candidate(L, gx * n, gy * n, fq[0], fq[1], flow + 2 * (size_t)g, &cost[g]);
          }
        }
      }
    }
  free(snap_f);
  free(snap_c);
}

/* Random search: F + O_rnd with O_rnd uniform in [-R_n, R_n]^2, kept only if
 * E_d decreases. The offset is drawn in units of 1/q pixel: integer pixels for
 * q = 1, the paper's subpixel offsets (with interpolated target colours) for
 * q = 2, 4; Rn is passed in those units. */
static void random_search(level_ctx *L, uint64_t seed, int flow_id, int level, int step, int Rn,
                          int32_t *flow, int32_t *cost) {
  int n = L->n, Gx = (L->W + n - 1) / n, Gy = (L->H + n - 1) / n;
  for (int gy = 0; gy < Gy; gy++)
    for (int gx = 0; gx < Gx; gx++) {
      int g = gy * Gx + gx;
      if (cost[g] == COST_UNSET) continue;
      int32_t d[2];
      ffo_rs_offset(seed, flow_id, level, step, gx, gy, Rn, d);
      int32_t *f = flow + 2 * (size_t)g;
      try_candidate(L, gx * n, gy * n, f[0] + d[0], f[1] + d[1], f, &cost[g]);
    }
}

/* Sec. 3.2, level transition: a grid point (gx, gy) of spacing n with both
 * coordinates even coincides with point (gx/2, gy/2) of spacing 2n and takes its
 * flow as a seed, with the cost re-evaluated on P^n_r. All other points start
 * without a flow and receive one in the first propagation pass. */
static void seed_level(level_ctx *L, const int32_t *flow_coarse, int32_t *flow, int32_t *cost) {
  int n = L->n, Gx = (L->W + n - 1) / n, Gy = (L->H + n - 1) / n;
  int Gxc = (L->W + 2 * n - 1) / (2 * n);
  for (int gy = 0; gy < Gy; gy++)
    for (int gx = 0; gx < Gx; gx++) {
      int g = gy * Gx + gx;
      flow[2 * g] = flow[2 * g + 1] = 0;
      cost[g] = COST_UNSET;
      if ((gx % 2) == 0 && (gy % 2) == 0) {
        const int32_t *fc = flow_coarse + 2 * ((size_t)(gy / 2) * Gxc + gx / 2);
        try_candidate(L, gx * n, gy * n, fc[0], fc[1], flow + 2 * g, &cost[g]);
      }
    }
}

/* One hierarchy level: optional seeding from the coarser level, then the
 * alternation P, RS, P, RS, P, RS, P (4 propagations, n_rs <= 3 random
 * searches, Sec. 3.1) with R_n = R * n (Sec. 3.2). Returns the number of E_d
 * evaluations (no candidate is skipped here). */
static int64_t search_level_q(const uint32_t *Cs, const uint32_t *const *Ct, int q, int W, int H,
                              int n, int r, const int32_t *flow_coarse, int tile, int n_rs, int R,
                              uint64_t seed, int flow_id, int32_t *flow, int32_t *cost,
                              const uint8_t *Ks, const uint8_t *Kt, int S) {
  level_ctx L = {Cs, Ct, W, H, n, r, q, 0, Ks, Kt, S};
  int level = 0;
  while ((1 << level) < n) level++;
  if (flow_coarse) seed_level(&L, flow_coarse, flow, cost);
  for (int s = 0; s < 4; s++) {
    prop_pass(&L, s, tile, flow, cost);
    if (s < 3 && s < n_rs) random_search(&L, seed, flow_id, level, s, R * n * q, flow, cost);
  }
  return L.evals;
}

int64_t ffo_search_level(const uint32_t *Cs, const uint32_t *Ct, int W, int H, int n, int r,
                         const int32_t *flow_coarse, int tile, int n_rs, int R, uint64_t seed,
                         int flow_id, int32_t *flow, int32_t *cost) {
  const uint32_t *Ct1[1] = {Ct};
  return search_level_q(Cs, Ct1, 1, W, H, n, r, flow_coarse, tile, n_rs, R, seed, flow_id, flow,
                        cost, NULL, NULL, 0);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4: outlier filtering.                                               */
/* Eq. 5 two-way check. Reading: the norm is Euclidean and compared strictly; */
/* with integer flows |.|^2 < eps^2 is used. Per pixel the squared errors     */
/* e_j = |F(p) + F^b_j(p + F(p))|^2 (e1, e2; may be NULL) and err_sum =       */
/* e1 + e2 (a diagnostic output). A target outside the image (never produced  */
/* by the search) fails the check; its errors are INT32_MAX.                  */
/* ------------------------------------------------------------------------ */
static int32_t clamp_i32(int64_t v) { return (int32_t)(v > INT32_MAX ? INT32_MAX : v); }

void ffo_consistency(const int32_t *F, const int32_t *Fb1, const int32_t *Fb2, int W, int H,
                     int eps, int q, uint8_t *valid_cc, int32_t *err_sum, int32_t *e1_out,
                     int32_t *e2_out) {
  /* flows in units of 1/q pixel: the backward flows are read at the pixel
   * nearest to the target (half rounded up), errors and eps in the same units */
  eps *= q;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      size_t p = (size_t)y * W + x;
      int qx = (int)floor_div((int64_t)q * x + F[2 * p] + q / 2, q);
      int qy = (int)floor_div((int64_t)q * y + F[2 * p + 1] + q / 2, q);
      if (qx < 0 || qx >= W || qy < 0 || qy >= H) {
        valid_cc[p] = 0;
        err_sum[p] = INT32_MAX;
        if (e1_out) e1_out[p] = INT32_MAX;
        if (e2_out) e2_out[p] = INT32_MAX;
        continue;
      }
      size_t q = (size_t)qy * W + qx;
      int64_t a0 = F[2 * p] + Fb1[2 * q], a1 = F[2 * p + 1] + Fb1[2 * q + 1];
      int64_t b0 = F[2 * p] + Fb2[2 * q], b1 = F[2 * p + 1] + Fb2[2 * q + 1];
      int64_t e1 = a0 * a0 + a1 * a1, e2 = b0 * b0 + b1 * b1;
      valid_cc[p] = (e1 < (int64_t)eps * eps) && (e2 < (int64_t)eps * eps);
      err_sum[p] = clamp_i32(e1 + e2);
      if (e1_out) e1_out[p] = clamp_i32(e1);
      if (e2_out) e2_out[p] = clamp_i32(e2);
    }
}

/* Is sqrt(a) + sqrt(b) < sqrt(c) + sqrt(d)?  Exact for integers 0 <= a..d < 2^28
 * (the squared errors of pixels that pass Eq. 5 are below eps^2 <= 10^6).
 * Both sides are non-negative, so squaring keeps the order:
 *   a + b + 2 sqrt(ab)  <  c + d + 2 sqrt(cd)
 *   <=>  u - v < t   with u = 2 sqrt(ab) = sqrt(4ab), v = sqrt(4cd), t = c + d - a - b.
 * u - v has the sign of 4ab - 4cd, which settles every case except two, where
 * one more squaring is needed:
 *   u < v, t < 0:   v - u > -t  <=>  v > u + (-t)  <=>  (4cd - 4ab - t^2) > 2(-t) u
 *   u > v, t > 0:   u - v <  t  <=>  u < v + t     <=>  (4ab - 4cd - t^2) < 2 t v
 * and a comparison  L > 2 s sqrt(Z)  (s >= 0) holds iff L > 0 and L^2 > 4 s^2 Z.
 * The products are formed in 128-bit integers. */
typedef __int128 i128;

static int gt_twice_sqrt(i128 L, i128 s, i128 Z) { /* L > 2 s sqrt(Z) */
  if (L <= 0) return 0;
  return L * L > 4 * s * s * Z;
}

int ffo_sqrt_sum_less(int64_t a, int64_t b, int64_t c, int64_t d) {
  const i128 X = (i128)4 * a * b, Y = (i128)4 * c * d, t = (i128)c + d - a - b;
  if (X == Y) return t > 0;
  if (X < Y) {
    if (t >= 0) return 1;
    return gt_twice_sqrt(Y - X - t * t, -t, X);
  }
  if (t <= 0) return 0;
  /* 4ab - 4cd - t^2 < 2 t sqrt(4cd)  <=>  not (4ab - 4cd - t^2 >= 2 t sqrt(4cd)) */
  {
    const i128 L = X - Y - t * t;
    if (L < 0) return 1;
    return L * L < 4 * t * t * Y;
  }
}

static int close3(const int32_t *F, size_t p, size_t q, int sub) { /* < 3 px, flows in 1/sub px */
  int64_t a = F[2 * p] - F[2 * q], b = F[2 * p + 1] - F[2 * q + 1];
  return a * a + b * b < 9ll * sub * sub;
}

/* Region filter. Pixels kept by the consistency check form regions: 4-connected
 * neighbours belong together when their flows differ by less than 3 px. A region
 * with fewer than s pixels is deleted if one of its pixels has a 4-neighbour that
 * the consistency check removed and whose (raw) flow is within 3 px of it, i.e.
 * the region could absorb that outlier by the same rule. */
void ffo_region_filter(const int32_t *F, const uint8_t *valid_cc, int W, int H, int s, int sub,
                       uint8_t *valid) {
  size_t N = (size_t)W * H;
  int32_t *label = malloc(sizeof(int32_t) * N), *queue = malloc(sizeof(int32_t) * N);
  static const int NB[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
  for (size_t p = 0; p < N; p++) label[p] = -1;
  memcpy(valid, valid_cc, N);
  for (size_t p0 = 0; p0 < N; p0++) {
    if (!valid_cc[p0] || label[p0] >= 0) continue;
    int head = 0, tail = 0, touches = 0;
    queue[tail++] = (int32_t)p0;
    label[p0] = (int32_t)p0;
    while (head < tail) {
      int p = queue[head++], x = p % W, y = p / W;
      for (int k = 0; k < 4; k++) {
        int xx = x + NB[k][0], yy = y + NB[k][1];
        if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
        size_t q = (size_t)yy * W + xx;
        if (!close3(F, p, q, sub)) continue;
        if (!valid_cc[q]) {
          touches = 1;
          continue;
        }
        if (label[q] < 0) {
          label[q] = (int32_t)p0;
          queue[tail++] = (int32_t)q;
        }
      }
    }
    if (tail < s && touches)
      for (int k = 0; k < tail; k++) valid[queue[k]] = 0;
  }
  free(label);
  free(queue);
}

/* Sec. 3.5 sparsification. Aligned 3x3 blocks (partial blocks at the right and
 * bottom edge included); a block with at least e surviving pixels keeps the one
 * for which the sum of its two consistency-check errors |.| (Eq. 5), i.e.
 * sqrt(e1) + sqrt(e2), is the smallest, the first in raster order within the
 * block on ties. Output rows (x, y, dx, dy) in block raster order; mask marks
 * them. Returns the number of rows. */
int ffo_sparsify(const uint8_t *valid, const int32_t *e1, const int32_t *e2, const int32_t *F,
                 int W, int H, int e, int32_t *sparse, uint8_t *mask) {
  int cnt_out = 0;
  memset(mask, 0, (size_t)W * H);
  for (int by = 0; by < (H + 2) / 3; by++)
    for (int bx = 0; bx < (W + 2) / 3; bx++) {
      int cnt = 0, best = -1;
      for (int y = 3 * by; y < imin(3 * by + 3, H); y++)
        for (int x = 3 * bx; x < imin(3 * bx + 3, W); x++) {
          int p = y * W + x;
          if (!valid[p]) continue;
          cnt++;
          if (best < 0 || ffo_sqrt_sum_less(e1[p], e2[p], e1[best], e2[best])) best = p;
        }
      if (cnt >= e && best >= 0) {
        mask[best] = 1;
        sparse[4 * cnt_out] = best % W;
        sparse[4 * cnt_out + 1] = best / W;
        sparse[4 * cnt_out + 2] = F[2 * best];
        sparse[4 * cnt_out + 3] = F[2 * best + 1];
        cnt_out++;
      }
    }
  return cnt_out;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1 (Table 1, "k=3+median"): the raw forward field filtered by a median */
/* weighted by the matching error. Reading (the paper gives neither window nor  */
/* weights): the matching error of pixel p is E(p) = E_d(P_r(p), P_r(p + F(p)))  */
/* at full resolution (census of both frames with spacing 1, taps clamped);     */
/* the weight w(q) = floor(2^16 / (1 + E(q))); the window holds the in-image    */
/* pixels q with max(|qx - px|, |qy - py|) <= rho; each flow component takes    */
/* the weighted lower median: the smallest value v with                        */
/* 2 * (sum of the weights of samples <= v) >= (sum of all weights).           */
/* ------------------------------------------------------------------------ */
void ffo_match_errors(const uint8_t *I1, const uint8_t *I2, const int32_t *F, int W, int H, int r,
                      int32_t *E) {
  size_t N = (size_t)W * H;
  uint32_t *C1 = malloc(sizeof(uint32_t) * N), *C2 = malloc(sizeof(uint32_t) * N);
  ffo_census(I1, W, H, 1, C1);
  ffo_census(I2, W, H, 1, C2);
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      size_t p = (size_t)y * W + x;
      E[p] = ffo_patch_cost(C1, C2, W, H, 1, r, x, y, x + F[2 * p], y + F[2 * p + 1]);
    }
  free(C1);
  free(C2);
}

void ffo_weighted_median(const int32_t *F, const int32_t *E, int W, int H, int rho, int32_t *out) {
  int cap = (2 * rho + 1) * (2 * rho + 1);
  int32_t *val = malloc(sizeof(int32_t) * cap);
  int64_t *wt = malloc(sizeof(int64_t) * cap);
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++)
      for (int comp = 0; comp < 2; comp++) {
        int m = 0;
        int64_t total = 0;
        for (int yy = y - rho; yy <= y + rho; yy++)
          for (int xx = x - rho; xx <= x + rho; xx++) {
            if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
            size_t q = (size_t)yy * W + xx;
            val[m] = F[2 * q + comp];
            wt[m] = 65536 / (1 + (int64_t)E[q]);
            total += wt[m];
            m++;
          }
        for (int i = 1; i < m; i++) /* insertion sort by value */
          for (int j = i; j > 0 && val[j - 1] > val[j]; j--) {
            int32_t tv = val[j];
            val[j] = val[j - 1];
            val[j - 1] = tv;
            int64_t tw = wt[j];
            wt[j] = wt[j - 1];
            wt[j - 1] = tw;
          }
        int64_t cum = 0;
        int32_t med = val[m - 1];
        for (int i = 0; i < m; i++) {
          cum += wt[i];
          if (2 * cum >= total) {
            med = val[i];
            break;
          }
        }
        out[2 * ((size_t)y * W + x) + comp] = med;
      }
  free(val);
  free(wt);
}

/* ------------------------------------------------------------------------ */
/* Whole pipeline (Fig. 2 and Sec. 3.4/3.5): three flow fields (forward with   */
/* radius r, backward with r, backward with r2), each from its own kd tree,   */
/* then consistency check, region filter and sparsification.                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int k, r, r2, leaf, R, eps, e, s, tile, n_rs, K;
  int color; /* 0: the RGB channels; 1: integer CIELab (Sec. 3.1 / 3.3) */
  int subpel; /* flows in units of 1/subpel pixel: 1, 2 or 4 (Sec. 3.1 subpixel search) */
  uint64_t seed;
} ffo_params;

typedef struct {
  const uint8_t *src, *tgt;
  uint32_t **Cs;         /* source census per level 0..k (phase 0) */
  uint32_t *(*Ct)[16];   /* target census per level and subpixel phase */
  int W, H, r, flow_id;
  const ffo_params *P;
  const int32_t *proposals;
  int32_t *flow_out; /* [H][W][2] */
  int64_t evals;
  /* S > 0: the SIFT flow data term, level-lv colours Ks[lv] (source) and Kt[lv] */
  uint8_t **Ks, **Kt;
  int S;
} flow_job;

static void *run_flow(void *arg) {
  flow_job *J = arg;
  const ffo_params *P = J->P;
  int W = J->W, H = J->H, N = W * H, ntop = 1 << P->k;
  int32_t *tf = malloc(sizeof(int32_t) * NFEAT * (size_t)N);
  ffo_wht_features(J->tgt, W, H, J->r, NULL, 0, tf);
  int Gx = (W + ntop - 1) / ntop, Gy = (H + ntop - 1) / ntop;
  int32_t *flow = malloc(sizeof(int32_t) * 2 * (size_t)Gx * Gy);
  int32_t *cost = malloc(sizeof(int32_t) * (size_t)Gx * Gy);
  int q = P->subpel;
  int S = J->S;
  J->evals = kd_init_q(tf, J->src, W, H, J->r, P->leaf, S ? NULL : J->Cs[P->k],
                       S ? NULL : (const uint32_t *const *)J->Ct[P->k], q, ntop, J->proposals,
                       J->proposals ? P->K : 0, flow, cost, S ? J->Ks[P->k] : NULL,
                       S ? J->Kt[P->k] : NULL, S);
  free(tf);
  J->evals += search_level_q(S ? NULL : J->Cs[P->k], S ? NULL : (const uint32_t *const *)J->Ct[P->k],
                             q, W, H, ntop, J->r, NULL, P->tile, P->n_rs, P->R, P->seed, J->flow_id,
                             flow, cost, S ? J->Ks[P->k] : NULL, S ? J->Kt[P->k] : NULL, S);
  for (int lv = P->k - 1; lv >= 0; lv--) {
    int n = 1 << lv;
    int gx = (W + n - 1) / n, gy = (H + n - 1) / n;
    int32_t *f2 = malloc(sizeof(int32_t) * 2 * (size_t)gx * gy);
    int32_t *c2 = malloc(sizeof(int32_t) * (size_t)gx * gy);
    J->evals += search_level_q(S ? NULL : J->Cs[lv], S ? NULL : (const uint32_t *const *)J->Ct[lv],
                               q, W, H, n, J->r, flow, P->tile, P->n_rs, P->R, P->seed, J->flow_id,
                               f2, c2, S ? J->Ks[lv] : NULL, S ? J->Kt[lv] : NULL, S);
    free(flow);
    free(cost);
    flow = f2;
    cost = c2;
  }
  memcpy(J->flow_out, flow, sizeof(int32_t) * 2 * (size_t)N);
  free(flow);
  free(cost);
  return NULL;
}

/* I1, I2: uint8 [H][W][3]. Outputs (all caller-allocated):
 *   flows   int32 [3][H][W][2]  forward, backward (r), backward (r2)
 *   valid   uint8 [H][W]        after consistency check and region filter
 *   err_sum int32 [H][W]
 *   sparse  int32 [ceil(W/3)*ceil(H/3)][4], mask uint8 [H][W]
 * proposals: NULL or int32 [Gy][Gx][K][2] at the coarsest grid (forward flow
 * only). threads > 1 runs the three flows concurrently. Returns the sparse
 * count; evals (optional) receives the number of E_d evaluations. */
int ffo_flow_fields(const uint8_t *I1_in, const uint8_t *I2_in, int W, int H,
                    const ffo_params *P, const int32_t *proposals, int threads, int32_t *flows,
                    uint8_t *valid, int32_t *err_sum, int32_t *sparse, uint8_t *mask,
                    int64_t *evals) {
  size_t N = (size_t)W * H;
  /* the colour space of every later step: the input channels or CIELab */
  uint8_t *lab1 = NULL, *lab2 = NULL;
  const uint8_t *I1 = I1_in, *I2 = I2_in;
  if (P->color == 1) {
    lab1 = malloc(N * 3);
    lab2 = malloc(N * 3);
    ffo_rgb_to_lab(I1_in, W, H, lab1);
    ffo_rgb_to_lab(I2_in, W, H, lab2);
    I1 = lab1;
    I2 = lab2;
  }
  int nl = P->k + 1, q = P->subpel, nph = q * q;
  /* census per frame, level and subpixel phase (phase 0 = the plain census) */
  uint32_t *C1[16][16], *C2[16][16], *C1s[16], *C2s[16];
  uint8_t *sm = malloc(N * 3);
  for (int lv = 0; lv < nl; lv++) {
    int n = 1 << lv;
    for (int f = 0; f < 2; f++) {
      ffo_smooth(f == 0 ? I1 : I2, W, H, n, sm);
      for (int ph = 0; ph < nph; ph++) {
        uint32_t *c = malloc(sizeof(uint32_t) * N);
        if (ph == 0) ffo_census(sm, W, H, n, c);
        else ffo_census_subpel(sm, W, H, n, q, ph % q, ph / q, c);
        (f == 0 ? C1 : C2)[lv][ph] = c;
      }
    }
    C1s[lv] = C1[lv][0];
    C2s[lv] = C2[lv][0];
  }
  free(sm);
  flow_job J[3] = {
      {I1, I2, C1s, C2, W, H, P->r, 0, P, proposals, flows, 0, NULL, NULL, 0},
      {I2, I1, C2s, C1, W, H, P->r, 1, P, NULL, flows + 2 * N, 0, NULL, NULL, 0},
      {I2, I1, C2s, C1, W, H, P->r2, 2, P, NULL, flows + 4 * N, 0, NULL, NULL, 0},
  };
  if (threads > 1) {
    pthread_t th[3];
    for (int i = 0; i < 3; i++) pthread_create(&th[i], NULL, run_flow, &J[i]);
    for (int i = 0; i < 3; i++) pthread_join(th[i], NULL);
  } else {
    for (int i = 0; i < 3; i++) run_flow(&J[i]);
  }
  for (int lv = 0; lv < nl; lv++)
    for (int ph = 0; ph < nph; ph++) {
      free(C1[lv][ph]);
      free(C2[lv][ph]);
    }
  uint8_t *vcc = malloc(N);
  int32_t *e1 = malloc(sizeof(int32_t) * N), *e2 = malloc(sizeof(int32_t) * N);
  ffo_consistency(flows, flows + 2 * N, flows + 4 * N, W, H, P->eps, q, vcc, err_sum, e1, e2);
  ffo_region_filter(flows, vcc, W, H, P->s, q, valid);
  free(vcc);
  if (evals) *evals = J[0].evals + J[1].evals + J[2].evals;
  int n = ffo_sparsify(valid, e1, e2, flows, W, H, P->e, sparse, mask);
  free(e1);
  free(e2);
  free(lab1);
  free(lab2);
  return n;
}

/* Level search and kd initialisation with the SIFT flow data term (Sec. 3.3):
 * the census steps above with E_d on the level-n colours Ks (source frame) and
 * Kt (target frame), S channels in S/3 groups (ffo_sift_colors), q = 1. */
int64_t ffo_sift_kd_init(const int32_t *tgt_feat, const uint8_t *src_img, int W, int H, int r,
                         int leaf, const uint8_t *Ks, const uint8_t *Kt, int S, int n,
                         int32_t *flow, int32_t *cost) {
  return kd_init_q(tgt_feat, src_img, W, H, r, leaf, NULL, NULL, 1, n, NULL, 0, flow, cost, Ks,
                   Kt, S);
}

int64_t ffo_sift_search_level(const uint8_t *Ks, const uint8_t *Kt, int S, int W, int H, int n,
                              int r, const int32_t *flow_coarse, int tile, int n_rs, int R,
                              uint64_t seed, int flow_id, int32_t *flow, int32_t *cost) {
  return search_level_q(NULL, NULL, 1, W, H, n, r, flow_coarse, tile, n_rs, R, seed, flow_id, flow,
                        cost, Ks, Kt, S);
}

/* The whole path with the SIFT flow data term (Sec. 3.3, Sec. 5 KITTI): SIFT
 * vectors of both input frames; colours with basis B1 (S1 channels) for the
 * forward and first backward flow, with B2 (S2 channels) for the second
 * backward flow (radius r2); per level the colour groups smoothed like I^n
 * (Sec. 3.2); the kd trees over WHT features as in ffo_flow_fields (CIELab
 * when P->color = 1); then the same consistency check, region filter and
 * sparsification. P->subpel and P->K are ignored (integer flows, no proposals).
 * B*: int16 [S][128], off*: int32 [S] (ffo_sift_pca_offset). Outputs as
 * ffo_flow_fields. */
int ffo_sift_flow_fields(const uint8_t *I1_in, const uint8_t *I2_in, int W, int H,
                         const ffo_params *P, const int16_t *B1, const int32_t *off1, int S1,
                         const int16_t *B2, const int32_t *off2, int S2, int threads,
                         int32_t *flows, uint8_t *valid, int32_t *err_sum, int32_t *sparse,
                         uint8_t *mask, int64_t *evals) {
  size_t N = (size_t)W * H;
  uint8_t *lab1 = NULL, *lab2 = NULL;
  const uint8_t *I1 = I1_in, *I2 = I2_in;
  if (P->color == 1) {
    lab1 = malloc(N * 3);
    lab2 = malloc(N * 3);
    ffo_rgb_to_lab(I1_in, W, H, lab1);
    ffo_rgb_to_lab(I2_in, W, H, lab2);
    I1 = lab1;
    I2 = lab2;
  }
  int nl = P->k + 1;
  uint8_t *d1 = malloc(N * SIFT_DIM), *d2 = malloc(N * SIFT_DIM);
  ffo_sift_descriptors(I1_in, W, H, d1);
  ffo_sift_descriptors(I2_in, W, H, d2);
  /* colours [set][frame][level]: set 0 = (B1, S1), set 1 = (B2, S2) */
  uint8_t *K[2][2][16];
  const int16_t *Bs[2] = {B1, B2};
  const int32_t *offs[2] = {off1, off2};
  int Ss[2] = {S1, S2};
  for (int c = 0; c < 2; c++)
    for (int f = 0; f < 2; f++) {
      size_t bytes = N * (size_t)Ss[c];
      uint8_t *full = malloc(bytes);
      ffo_sift_colors(f == 0 ? d1 : d2, W, H, Bs[c], offs[c], Ss[c], full);
      for (int lv = 0; lv < nl; lv++) {
        K[c][f][lv] = malloc(bytes);
        for (int g = 0; g < Ss[c] / 3; g++)
          ffo_smooth(full + (size_t)g * N * 3, W, H, 1 << lv, K[c][f][lv] + (size_t)g * N * 3);
      }
      free(full);
    }
  free(d1);
  free(d2);
  flow_job J[3] = {
      {I1, I2, NULL, NULL, W, H, P->r, 0, P, NULL, flows, 0, K[0][0], K[0][1], S1},
      {I2, I1, NULL, NULL, W, H, P->r, 1, P, NULL, flows + 2 * N, 0, K[0][1], K[0][0], S1},
      {I2, I1, NULL, NULL, W, H, P->r2, 2, P, NULL, flows + 4 * N, 0, K[1][1], K[1][0], S2},
  };
  ffo_params P1 = *P;
  P1.subpel = 1;
  P1.K = 0;
  for (int i = 0; i < 3; i++) J[i].P = &P1;
  if (threads > 1) {
    pthread_t th[3];
    for (int i = 0; i < 3; i++) pthread_create(&th[i], NULL, run_flow, &J[i]);
    for (int i = 0; i < 3; i++) pthread_join(th[i], NULL);
  } else {
    for (int i = 0; i < 3; i++) run_flow(&J[i]);
  }
  for (int c = 0; c < 2; c++)
    for (int f = 0; f < 2; f++)
      for (int lv = 0; lv < nl; lv++) free(K[c][f][lv]);
  uint8_t *vcc = malloc(N);
  int32_t *e1 = malloc(sizeof(int32_t) * N), *e2 = malloc(sizeof(int32_t) * N);
  ffo_consistency(flows, flows + 2 * N, flows + 4 * N, W, H, P->eps, 1, vcc, err_sum, e1, e2);
  ffo_region_filter(flows, vcc, W, H, P->s, 1, valid);
  free(vcc);
  if (evals) *evals = J[0].evals + J[1].evals + J[2].evals;
  int n = ffo_sparsify(valid, e1, e2, flows, W, H, P->e, sparse, mask);
  free(e1);
  free(e2);
  free(lab1);
  free(lab2);
  return n;
}
