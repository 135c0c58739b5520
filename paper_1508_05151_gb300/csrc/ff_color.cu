// Sec. 3.1 / 3.3: the paper computes the WHT features and the census transform
// in CIELab. This is an integer CIELab of 8-bit sRGB (D65 white, the sRGB
// primaries of IEC 61966-2-1), exact after its 256-entry decoding table:
//   lin   = round(65536 g(v / 255)), g the sRGB decoding curve (1.0 = 65536)
//   t_i   = (row_i . lin + 8192) >> 14, row_i = i-th row of the sRGB->XYZ matrix
//           divided by the white point's component, in Q14, each row rounded to
//           sum to exactly 16384 (the residual on its largest entry), so a grey
//           pixel gives t_X = t_Y = t_Z
//   f(t)  = floor(65536 cbrt(t / 65536)) (the largest y with y^3 <= t 2^32) when
//           t / 65536 > (6/29)^3, else t / (3 (6/29)^2) + 4/29 in Q16, rounded
//   L, a, b = 116 f_Y - 16, 500 (f_X - f_Y), 200 (f_Y - f_Z), stored as uint8
//           L * 255 / 100, a + 128, b + 128 (rounded half up, clamped).
#include <math.h>

#include <mutex>

#include "ff_internal.cuh"

namespace ff {

struct LabTables {
  int32_t lin[256];
  int32_t m[9];
};

// The decoding table and the normalised matrix, computed once on the host.
static const LabTables &lab_tables() {
  static LabTables t;
  static std::once_flag once;
  std::call_once(once, [] {
    for (int v = 0; v < 256; v++) {
      const double c = v / 255.0;
      const double g = c <= 0.04045 ? c / 12.92 : pow((c + 0.055) / 1.055, 2.4);
      t.lin[v] = (int32_t)floor(g * 65536.0 + 0.5);
    }
    // sRGB -> XYZ (IEC 61966-2-1), rows over the D65 white's X, Y, Z
    const double M[3][3] = {{0.4124, 0.3576, 0.1805}, {0.2126, 0.7152, 0.0722},
                            {0.0193, 0.1192, 0.9505}};
    for (int i = 0; i < 3; i++) {
      const double white = M[i][0] + M[i][1] + M[i][2];
      int sum = 0, big = 0;
      for (int j = 0; j < 3; j++) {
        t.m[3 * i + j] = (int32_t)floor(M[i][j] / white * 16384.0 + 0.5);
        sum += t.m[3 * i + j];
        if (M[i][j] > M[i][big]) big = j;
      }
      t.m[3 * i + big] += 16384 - sum;
    }
  });
  return t;
}

// f(t) of the Lab transfer in Q16, t in [0, 65536].
__device__ __forceinline__ int32_t lab_f(int32_t t) {
  if ((long long)t * 24389 > 216ll * 65536) {  // t / 65536 > (6/29)^3: cube root
    const unsigned long long target = (unsigned long long)t << 32;
    long long y = (long long)cbrt((double)target);  // estimate, then the exact integer
    while (y > 0 && (unsigned long long)(y * y * y) > target) y--;
    while ((unsigned long long)((y + 1) * (y + 1) * (y + 1)) <= target) y++;
    return (int32_t)y;
  }
  return (int32_t)((29ll * 841 * t + 108ll * 4 * 65536 + 1566) / 3132);  // positive: / floors
}

// round(num / den) half up for den > 0, num of any sign, plus offset, clamped to a byte
__device__ __forceinline__ uint8_t lab_byte(long long num, long long den, int offset) {
  long long q = 2 * num + den, d2 = 2 * den;
  long long v = q >= 0 ? q / d2 : -((-q + d2 - 1) / d2);
  v += offset;
  return (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
}

__global__ void __launch_bounds__(256) k_rgb_to_lab(const uint8_t *__restrict__ img, int N,
                                                    LabTables tab, uint8_t *__restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int c0 = tab.lin[img[3 * p]], c1 = tab.lin[img[3 * p + 1]], c2 = tab.lin[img[3 * p + 2]];
  int32_t f[3];
#pragma unroll
  for (int i = 0; i < 3; i++) {
    const long long t =
        ((long long)tab.m[3 * i] * c0 + (long long)tab.m[3 * i + 1] * c1 + (long long)tab.m[3 * i + 2] * c2 + 8192) >> 14;
    f[i] = lab_f((int32_t)t);
  }
  out[3 * p] = lab_byte((116ll * f[1] - 16ll * 65536) * 255, 100ll * 65536, 0);
  out[3 * p + 1] = lab_byte(500ll * (f[0] - f[1]), 65536, 128);
  out[3 * p + 2] = lab_byte(200ll * (f[1] - f[2]), 65536, 128);
}

ff_status launch_rgb_to_lab(const uint8_t *img, int W, int H, uint8_t *out, cudaStream_t st) {
  const int N = W * H;
  if (N <= 0) return FF_OK;
  k_rgb_to_lab<<<(N + 255) / 256, 256, 0, st>>>(img, N, lab_tables(), out);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

}  // namespace ff

using namespace ff;

extern "C" ff_status ff_rgb_to_lab(const uint8_t *img, int W, int H, uint8_t *out, void *stream) {
  FF_TRY(check_shape(W, H));
  if (!img || !out) return FF_ERR_INVALID_ARG;
  return launch_rgb_to_lab(img, W, H, out, (cudaStream_t)stream);
}
