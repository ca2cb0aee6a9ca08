// Multi-resolution pyramid (factor 2, Ploner et al. Sec. 2.1; the validity
// is downsampled "in the same way", Sec. 2.2), displacement prolongation
// between levels, and depth padding of the device volumes.
//
// Box mean over 2 samples per axis; an odd size rounds up and the missing
// sample repeats the edge sample.  The 8 (4, 2) float samples are added in
// double, which is exact for float inputs of similar magnitude, and the mean
// is rounded once to float.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace octmc {
namespace {

constexpr int kThreads = 256;

__global__ void pad_depth_kernel(float* vol, int64_t columns, int d, int dp) {
  const int padn = dp - d;
  const int64_t n = columns * padn;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / padn;
    const int k = d + (int)(e % padn);
    vol[col * dp + k] = vol[col * dp + d - 1];
  }
}

__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_float(__half v) { return __half2float(v); }

template <typename T>
__global__ void unpad_depth_kernel(const T* vol, int64_t columns, int d, int dp, float* out) {
  const int64_t n = columns * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / d;
    out[e] = to_float(vol[col * dp + (e % d)]);
  }
}

// float32 -> 16-bit storage type, round to nearest even.
__device__ __forceinline__ void store_as(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_as(__half* p, float v) { *p = __float2half_rn(v); }

template <typename T>
__global__ void convert_kernel(const float* __restrict__ in, T* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    store_as(out + e, in[e]);
}

// One thread per output sample (i2, j2, k2) including the depth pad.
__global__ void pyr_volume_kernel(const float* __restrict__ in, int w, int h, int d, int dp,
                                  float* __restrict__ out, int w2, int h2, int d2, int dp2) {
  const int64_t n = (int64_t)w2 * h2 * dp2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / dp2;
    int k2 = (int)(e % dp2);
    if (k2 >= d2) k2 = d2 - 1;  // depth pad repeats the last sample
    const int i2 = (int)(col % w2), j2 = (int)(col / w2);
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const int j = min(2 * j2 + b, h - 1);
#pragma unroll
      for (int a = 0; a < 2; a++) {
        const int i = min(2 * i2 + a, w - 1);
        const float* c = in + ((int64_t)j * w + i) * dp;
        s += (double)c[min(2 * k2, d - 1)] + (double)c[min(2 * k2 + 1, d - 1)];
      }
    }
    out[e] = (float)(s * 0.125);
  }
}

__global__ void pyr_image_kernel(const float* __restrict__ in, int w, int h, float* __restrict__ out) {
  const int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
  const int64_t n = (int64_t)w2 * h2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i2 = (int)(e % w2), j2 = (int)(e / w2);
    const int i0 = 2 * i2, i1 = min(2 * i2 + 1, w - 1), j0 = 2 * j2, j1 = min(2 * j2 + 1, h - 1);
    const double s = (double)in[(int64_t)j0 * w + i0] + (double)in[(int64_t)j0 * w + i1] +
                     (double)in[(int64_t)j1 * w + i0] + (double)in[(int64_t)j1 * w + i1];
    out[e] = (float)(s * 0.25);
  }
}

__global__ void pyr_line_kernel(const float* __restrict__ in, int n, float* __restrict__ out) {
  const int n2 = (n + 1) / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += gridDim.x * blockDim.x)
    out[e] = (float)(((double)in[2 * e] + (double)in[min(2 * e + 1, n - 1)]) * 0.5);
}

// Fine A-scan i sits at (i - 1/2)/2 on the coarse grid (box-filter centres);
// bilinear there with the coordinate clamped into the grid, value doubled
// because the pixel unit halves.
__global__ void prolong_kernel(const double* __restrict__ coarse, int wc, int hc,
                               double* __restrict__ fine, int wf, int hf) {
  const int64_t pf = (int64_t)wf * hf, pc = (int64_t)wc * hc;
  const int64_t n = 6 * pf;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int plane = (int)(e / pf);
    const int64_t q = e % pf;
    const int i = (int)(q % wf), j = (int)(q / wf);
    const double x = fmin(fmax(0.5 * i - 0.25, 0.0), (double)(wc - 1));
    const double y = fmin(fmax(0.5 * j - 0.25, 0.0), (double)(hc - 1));
    const int x0 = (int)x, y0 = (int)y;  // x, y >= 0: truncation is floor
    const int x1 = min(x0 + 1, wc - 1), y1 = min(y0 + 1, hc - 1);
    const double fx = x - x0, fy = y - y0;
    const double* c = coarse + plane * pc;
    const double top = c[(int64_t)y0 * wc + x0] + fx * (c[(int64_t)y0 * wc + x1] - c[(int64_t)y0 * wc + x0]);
    const double bot = c[(int64_t)y1 * wc + x0] + fx * (c[(int64_t)y1 * wc + x1] - c[(int64_t)y1 * wc + x0]);
    fine[e] = 2.0 * (top + fy * (bot - top));
  }
}

inline unsigned grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 65535) b = 65535;
  return (unsigned)b;
}

}  // namespace

cudaError_t launch_pad_depth(float* vol, int64_t columns, int d, int dp, cudaStream_t s) {
  if (dp == d) return cudaSuccess;
  pad_depth_kernel<<<grid_for(columns * (dp - d)), kThreads, 0, s>>>(vol, columns, d, dp);
  return cudaGetLastError();
}

cudaError_t launch_unpad_depth(const void* vol, int dtype, int64_t columns, int d, int dp, float* out,
                               cudaStream_t s) {
  const unsigned g = grid_for(columns * d);
  if (dtype == OCTMC_BF16)
    unpad_depth_kernel<<<g, kThreads, 0, s>>>(static_cast<const __nv_bfloat16*>(vol), columns, d, dp, out);
  else if (dtype == OCTMC_F16)
    unpad_depth_kernel<<<g, kThreads, 0, s>>>(static_cast<const __half*>(vol), columns, d, dp, out);
  else
    unpad_depth_kernel<<<g, kThreads, 0, s>>>(static_cast<const float*>(vol), columns, d, dp, out);
  return cudaGetLastError();
}

cudaError_t launch_convert(const float* in, void* out, int dtype, int64_t n, cudaStream_t s) {
  const unsigned g = grid_for(n);
  if (dtype == OCTMC_BF16)
    convert_kernel<<<g, kThreads, 0, s>>>(in, static_cast<__nv_bfloat16*>(out), n);
  else if (dtype == OCTMC_F16)
    convert_kernel<<<g, kThreads, 0, s>>>(in, static_cast<__half*>(out), n);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_pyr_volume(const float* in, int w, int h, int d, int dp, float* out, int w2, int h2,
                              int d2, int dp2, cudaStream_t s) {
  pyr_volume_kernel<<<grid_for((int64_t)w2 * h2 * dp2), kThreads, 0, s>>>(in, w, h, d, dp, out, w2, h2,
                                                                          d2, dp2);
  return cudaGetLastError();
}

cudaError_t launch_pyr_image(const float* in, int w, int h, float* out, cudaStream_t s) {
  pyr_image_kernel<<<grid_for((int64_t)((w + 1) / 2) * ((h + 1) / 2)), kThreads, 0, s>>>(in, w, h, out);
  return cudaGetLastError();
}

cudaError_t launch_pyr_line(const float* in, int n, float* out, cudaStream_t s) {
  pyr_line_kernel<<<grid_for((n + 1) / 2), kThreads, 0, s>>>(in, n, out);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const double* coarse, int wc, int hc, double* fine, int wf, int hf,
                           cudaStream_t s) {
  prolong_kernel<<<grid_for(6LL * wf * hf), kThreads, 0, s>>>(coarse, wc, hc, fine, wf, hf);
  return cudaGetLastError();
}

}  // namespace octmc
