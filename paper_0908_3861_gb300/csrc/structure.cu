// Scale-map estimation: an edge-following ellipse per pixel from the image's
// structure tensor, the input of the filter's ellipse scale kind.  The paper
// leaves the scale map to other work (Sec. 8); this is the reading taken here:
//
//   gradient by central differences (zero outside the image),
//   J = G_rho * (g g^T), a separable sampled Gaussian (|k| <= ceil(3 rho),
//     weights normalised to 1, zero outside the image),
//   l1 >= l2 the eigenvalues of J, coherence ((l1 - l2) / (l1 + l2 + eps))^2,
//   ellipse: size sigma0, elongation 1 + (e_max - 1) coherence, major axis the
//     eigenvector of l2 as (cos t, sin t), sin t >= 0; (1, 0) where l1 == l2.
//
// Kernels: products (gx^2, gx gy, gy^2 in binary32), the row pass of the
// Gaussian, and the column pass fused with the eigen-analysis (binary64) and
// the output (float4 per pixel).  All memory-bound stencils.
#include <cmath>
#include <vector>

#include "abf_internal.cuh"

namespace abf {

constexpr int kMaxGaussTaps = 63;  // rho <= 10

struct GaussTaps {
  int r;
  float w[kMaxGaussTaps];
};

template <typename TIn>
__device__ __forceinline__ float pix(const TIn* f, size_t pitch, int W, int H, int x, int y) {
  if (x < 0 || x >= W || y < 0 || y >= H) return 0.0f;
  return (float)reinterpret_cast<const TIn*>(reinterpret_cast<const char*>(f) + (size_t)y * pitch)[x];
}

template <typename TIn>
__global__ void st_products_kernel(const TIn* __restrict__ f, size_t pitch, int W, int H, float* __restrict__ j11,
                                   float* __restrict__ j12, float* __restrict__ j22) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  const float gx = 0.5f * (pix(f, pitch, W, H, x + 1, y) - pix(f, pitch, W, H, x - 1, y));
  const float gy = 0.5f * (pix(f, pitch, W, H, x, y + 1) - pix(f, pitch, W, H, x, y - 1));
  const size_t i = (size_t)y * W + x;
  j11[i] = gx * gx;
  j12[i] = gx * gy;
  j22[i] = gy * gy;
}

// Row pass of the Gaussian on the three planes (a -> b).
__global__ void st_hblur_kernel(const float* __restrict__ a, float* __restrict__ b, int W, int H,
                                const GaussTaps taps) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, plane = blockIdx.z;
  if (x >= W) return;
  const float* row = a + (size_t)plane * W * H + (size_t)y * W;
  float acc = 0.0f;
  for (int k = -taps.r; k <= taps.r; ++k) {
    const int xx = x + k;
    if (xx >= 0 && xx < W) acc += taps.w[k + taps.r] * row[xx];
  }
  b[(size_t)plane * W * H + (size_t)y * W + x] = acc;
}

// Column pass, eigen-analysis and output.
__global__ void st_vblur_ellipse_kernel(const float* __restrict__ b, int W, int H, const GaussTaps taps,
                                        double sigma0, double e_max, float4* __restrict__ out, size_t out_pitch) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  float s[3] = {0.0f, 0.0f, 0.0f};
  for (int k = -taps.r; k <= taps.r; ++k) {
    const int yy = y + k;
    if (yy < 0 || yy >= H) continue;
    const float wk = taps.w[k + taps.r];
#pragma unroll
    for (int p = 0; p < 3; ++p) s[p] += wk * b[(size_t)p * W * H + (size_t)yy * W + x];
  }
  const double j11 = s[0], j12 = s[1], j22 = s[2];
  const double tr = j11 + j22;
  const double d = sqrt((j11 - j22) * (j11 - j22) + 4.0 * j12 * j12);
  const double l1 = 0.5 * (tr + d), l2 = 0.5 * (tr - d);
  const double q = (l1 - l2) / (l1 + l2 + 1e-12);
  const double coh = q * q;
  double ax = j12, ay = l2 - j11, bx = l2 - j22, by = j12;
  double vx, vy;
  if (bx * bx + by * by > ax * ax + ay * ay) {
    vx = bx;
    vy = by;
  } else {
    vx = ax;
    vy = ay;
  }
  const double n = sqrt(vx * vx + vy * vy);
  if (n == 0.0) {
    vx = 1.0;
    vy = 0.0;
  } else {
    vx /= n;
    vy /= n;
  }
  if (vy < 0.0 || (vy == 0.0 && vx < 0.0)) {
    vx = -vx;
    vy = -vy;
  }
  float4* orow = reinterpret_cast<float4*>(reinterpret_cast<char*>(out) + (size_t)y * out_pitch);
  orow[x] = make_float4((float)sigma0, (float)(1.0 + (e_max - 1.0) * coh), (float)vx, (float)vy);
}

static cudaError_t run_ellipses(const void* f, size_t pitch, int dtype, int W, int H, double rho, double sigma0,
                                double e_max, void* ws, void* out, size_t out_pitch, cudaStream_t st) {
  GaussTaps taps;
  taps.r = (int)std::ceil(3.0 * rho);
  std::vector<double> w(2 * taps.r + 1);
  double sum = 0.0;
  for (int k = -taps.r; k <= taps.r; ++k) sum += (w[k + taps.r] = std::exp(-(double)(k * k) / (2.0 * rho * rho)));
  for (int k = 0; k <= 2 * taps.r; ++k) taps.w[k] = (float)(w[k] / sum);
  float* a = (float*)ws;
  float* b = a + (size_t)3 * W * H;
  dim3 blk(256), grid((W + 255) / 256, H);
  float* j11 = a;
  float* j12 = a + (size_t)W * H;
  float* j22 = a + (size_t)2 * W * H;
  switch (dtype) {
    case ABF_U8: st_products_kernel<<<grid, blk, 0, st>>>((const uint8_t*)f, pitch, W, H, j11, j12, j22); break;
    case ABF_U16: st_products_kernel<<<grid, blk, 0, st>>>((const uint16_t*)f, pitch, W, H, j11, j12, j22); break;
    case ABF_F32: st_products_kernel<<<grid, blk, 0, st>>>((const float*)f, pitch, W, H, j11, j12, j22); break;
    default: st_products_kernel<<<grid, blk, 0, st>>>((const double*)f, pitch, W, H, j11, j12, j22); break;
  }
  st_hblur_kernel<<<dim3(grid.x, H, 3), blk, 0, st>>>(a, b, W, H, taps);
  st_vblur_ellipse_kernel<<<grid, blk, 0, st>>>(b, W, H, taps, sigma0, e_max, (float4*)out, out_pitch);
  return cudaGetLastError();
}

}  // namespace abf

extern "C" {

size_t abf_ellipse_ws_bytes(int32_t width, int32_t height) {
  if (width < 1 || height < 1) return 0;
  return (size_t)6 * width * height * sizeof(float);
}

abf_status abf_estimate_ellipses(const void* d_f, size_t f_pitch, abf_dtype in_dtype, int32_t width, int32_t height,
                                 double rho, double sigma0, double e_max, void* d_ws, size_t ws_bytes, void* d_out,
                                 size_t out_pitch, cudaStream_t st) {
  if (!d_f || !d_ws || !d_out || width < 1 || height < 1 || height > 65535) return ABF_ERR_INVALID;
  if (in_dtype < ABF_U8 || in_dtype > ABF_F64) return ABF_ERR_INVALID;
  const size_t esz = in_dtype == ABF_U8 ? 1 : in_dtype == ABF_U16 ? 2 : in_dtype == ABF_F32 ? 4 : 8;
  if (f_pitch < (size_t)width * esz || out_pitch < (size_t)width * 16 || (out_pitch & 15) ||
      ((uintptr_t)d_out & 15) || ((uintptr_t)d_ws & 3))
    return ABF_ERR_INVALID;
  if (!(rho > 0.0) || rho > 10.0 || !(sigma0 > 0.0) || !(e_max >= 1.0) || !std::isfinite(sigma0) ||
      !std::isfinite(e_max))
    return ABF_ERR_INVALID;
  if (ws_bytes < abf_ellipse_ws_bytes(width, height)) return ABF_ERR_INVALID;
  return abf::run_ellipses(d_f, f_pitch, in_dtype, width, height, rho, sigma0, e_max, d_ws, d_out, out_pitch, st) ==
                 cudaSuccess
             ? ABF_OK
             : ABF_ERR_CUDA;
}

}  // extern "C"
