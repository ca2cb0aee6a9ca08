// Float64 vector kernels of the on-device L-BFGS (Ploner et al. Sec. 2.1:
// "gradient-based L-BFGS solver"): batched dot products with a fixed
// reduction order, linear combinations, differences and axpy.
#include "common.cuh"

namespace octmc {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 8;          // dot products per block row
constexpr int kMaxDotBlocks = 304; // blocks per chunk (2 per SM)

__device__ bool last_block_2d(unsigned* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// grid (G, chunks): block (bx, c) accumulates dots c*8 .. c*8+7 over a
// strided share of the n elements; chunk 0 also takes max|maxabs_of|.
// partials layout: [dot][G] and [kMaxDots][G] for the max.
__global__ void __launch_bounds__(kThreads) dots_kernel(const DotList L, int64_t n,
                                                        const double* __restrict__ maxabs_of,
                                                        double* partials, unsigned* counter,
                                                        double* out) {
  __shared__ double sm[(kChunk + 1) * (kThreads / 32)];
  const int G = gridDim.x;
  const int c0 = blockIdx.y * kChunk;
  double acc[kChunk + 1];
#pragma unroll
  for (int t = 0; t <= kChunk; t++) acc[t] = 0.0;
  const double* a[kChunk];
  const double* b[kChunk];
#pragma unroll
  for (int t = 0; t < kChunk; t++) {
    a[t] = (c0 + t < L.n) ? L.a[c0 + t] : nullptr;
    b[t] = (c0 + t < L.n) ? L.b[c0 + t] : nullptr;
  }
  const bool do_max = (blockIdx.y == 0) && maxabs_of;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < n; e += (int64_t)G * kThreads) {
#pragma unroll
    for (int t = 0; t < kChunk; t++)
      if (a[t]) acc[t] = fma(a[t][e], b[t][e], acc[t]);
    if (do_max) acc[kChunk] = fmax(acc[kChunk], fabs(maxabs_of[e]));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t <= kChunk; t++) {
    double v = acc[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_xor_sync(0xffffffffu, v, o);
      v = (t == kChunk) ? fmax(v, u) : v + u;
    }
    if (lane == 0) sm[t * (kThreads / 32) + warp] = v;
  }
  __syncthreads();
  if (threadIdx.x <= kChunk) {
    const int t = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; w++) {
      const double u = sm[t * (kThreads / 32) + w];
      v = (t == kChunk) ? fmax(v, u) : v + u;
    }
    if (t < kChunk && c0 + t < L.n) partials[(int64_t)(c0 + t) * G + blockIdx.x] = v;
    if (t == kChunk && blockIdx.y == 0) partials[(int64_t)kMaxDots * G + blockIdx.x] = v;
  }
  if (last_block_2d(counter)) {
    // the last block adds the partials of each dot: one warp per dot, lanes
    // take a fixed strided share of the blocks, then a butterfly
    for (int dd = warp; dd <= L.n; dd += kThreads / 32) {
      const bool is_max = (dd == L.n);
      const int64_t row = is_max ? kMaxDots : dd;
      double v = 0.0;
      for (int bx = lane; bx < G; bx += 32) {
        const double u = partials[row * G + bx];
        v = is_max ? fmax(v, u) : v + u;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmax(v, u) : v + u;
      }
      if (lane == 0) out[is_max ? kMaxDots : dd] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
  }
}

__global__ void lincomb_kernel(const LinComb C, int64_t n, double* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int v = 0; v < C.n; v++) s = fma(C.c[v], C.v[v][e], s);
    out[e] = s;
  }
}

__global__ void sub2_kernel(const double* __restrict__ x1, const double* __restrict__ x0,
                            const double* __restrict__ g1, const double* __restrict__ g0,
                            double* __restrict__ s, double* __restrict__ y, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    s[e] = x1[e] - x0[e];
    y[e] = g1[e] - g0[e];
  }
}

__global__ void axpy_kernel(const double* __restrict__ x, double a, const double* __restrict__ d,
                            double* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = fma(a, d[e], x[e]);
}

inline unsigned grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 4 * 152) b = 4 * 152;
  return (unsigned)b;
}

}  // namespace

// At least kPerThread elements per thread: every block ends in float64
// butterflies (slow on this GPU), so short vectors get few blocks.
constexpr int kPerThread = 8;
int dots_grid_blocks(int64_t n) {
  int64_t b = (n + (int64_t)kThreads * kPerThread - 1) / ((int64_t)kThreads * kPerThread);
  if (b < 1) b = 1;
  if (b > kMaxDotBlocks) b = kMaxDotBlocks;
  return (int)b;
}

cudaError_t launch_dots(const DotList& dl, int64_t n, const double* maxabs_of, double* partials,
                        unsigned* counter, double* out, cudaStream_t s) {
  const int G = dots_grid_blocks(n);
  const int chunks = dl.n > 0 ? (dl.n + kChunk - 1) / kChunk : 1;
  dots_kernel<<<dim3(G, chunks), kThreads, 0, s>>>(dl, n, maxabs_of, partials, counter, out);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(const LinComb& lc, int64_t n, double* out, cudaStream_t s) {
  lincomb_kernel<<<grid_for(n), kThreads, 0, s>>>(lc, n, out);
  return cudaGetLastError();
}

cudaError_t launch_sub2(const double* x1, const double* x0, const double* g1, const double* g0,
                        double* s_out, double* y_out, int64_t n, cudaStream_t st) {
  sub2_kernel<<<grid_for(n), kThreads, 0, st>>>(x1, x0, g1, g0, s_out, y_out, n);
  return cudaGetLastError();
}

cudaError_t launch_axpy(const double* x, double a, const double* d, double* out, int64_t n,
                        cudaStream_t s) {
  axpy_kernel<<<grid_for(n), kThreads, 0, s>>>(x, a, d, out, n);
  return cudaGetLastError();
}

}  // namespace octmc
