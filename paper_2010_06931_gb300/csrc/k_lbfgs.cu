// Vector kernels of the on-device L-BFGS (Ploner et al. Sec. 2.1:
// "gradient-based L-BFGS solver"): dot products of the history with probe
// vectors, the direction as a linear combination, pair differences and axpy.
//
// Everything is float64: the history pairs, the products with them (FMAs
// on doubles) and their sums.  Each thread sums a strided share of the
// elements, warps reduce with a fixed butterfly and blocks with fixed
// trees, so every result is deterministic.
#include "common.cuh"

namespace octmc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kHistChunk = 20;         // history vectors per block row
constexpr int kPerThread = 8;          // elements per thread (at least)
constexpr int kMaxDotBlocks = 8 * 152; // blocks per row

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

__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// grid (G, rows): block (bx, r) takes history vectors r*20 .. r*20+19 over
// a strided share of the n elements; row 0 also takes q0.q0, q1.q1 and
// max|q1| (the maximum on the bit patterns: exact, and NaN wins).
// partials layout: [output][G].
__global__ void __launch_bounds__(kThreads) hist_dots_kernel(const HistDots D, int64_t n, double* partials,
                                                             unsigned* counter, double* out) {
  __shared__ double sm[(2 * kHistChunk + 3) * kWarps];
  const int G = gridDim.x;
  const int k0 = blockIdx.y * kHistChunk;
  const int kn = min(kHistChunk, D.K - k0);  // <= 0 only in row 0 of an empty history
  const bool first = blockIdx.y == 0;
  const double* h[kHistChunk];
#pragma unroll
  for (int k = 0; k < kHistChunk; k++) h[k] = (k < kn) ? D.h[k0 + k] : nullptr;
  double a0[kHistChunk], a1[kHistChunk];
#pragma unroll
  for (int k = 0; k < kHistChunk; k++) a0[k] = a1[k] = 0.0;
  double qq0 = 0.0, qq1 = 0.0;
  unsigned long long mx = 0ull;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < n; e += (int64_t)G * kThreads) {
    const double v0 = D.q0 ? D.q0[e] : 0.0;
    const double g = D.q1 ? D.q1[e] : 0.0;
#pragma unroll
    for (int k = 0; k < kHistChunk; k++) {
      if (k < kn) {
        const double hv = h[k][e];
        a0[k] = fma(hv, v0, a0[k]);
        a1[k] = fma(hv, g, a1[k]);
      }
    }
    if (first) {
      qq0 = fma(v0, v0, qq0);
      qq1 = fma(g, g, qq1);
      mx = max(mx, abs_bits(g));
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kHistChunk; k++) {
    if (k < kn) {
      double u0 = a0[k], u1 = a1[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        u0 += __shfl_xor_sync(0xffffffffu, u0, o);
        u1 += __shfl_xor_sync(0xffffffffu, u1, o);
      }
      if (lane == 0) {
        sm[(2 * k) * kWarps + warp] = u0;
        sm[(2 * k + 1) * kWarps + warp] = u1;
      }
    }
  }
  if (first) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      qq0 += __shfl_xor_sync(0xffffffffu, qq0, o);
      qq1 += __shfl_xor_sync(0xffffffffu, qq1, o);
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
      sm[(2 * kHistChunk) * kWarps + warp] = qq0;
      sm[(2 * kHistChunk + 1) * kWarps + warp] = qq1;
      sm[(2 * kHistChunk + 2) * kWarps + warp] = __longlong_as_double((long long)mx);
    }
  }
  __syncthreads();
  const int nloc = 2 * max(kn, 0);
  for (int t = threadIdx.x; t < 2 * kHistChunk + 3; t += kThreads) {
    if (t < nloc) {
      double v = 0.0;
      for (int w = 0; w < kWarps; w++) v += sm[t * kWarps + w];
      partials[(int64_t)(2 * k0 + t) * G + blockIdx.x] = v;
    } else if (first && t >= 2 * kHistChunk) {
      const int x = t - 2 * kHistChunk;  // 0: q0.q0, 1: q1.q1, 2: max|q1|
      double v = 0.0;
      unsigned long long m = 0ull;
      for (int w = 0; w < kWarps; w++) {
        const double u = sm[t * kWarps + w];
        if (x == 2) m = max(m, (unsigned long long)__double_as_longlong(u));
        else v += u;
      }
      partials[(int64_t)(2 * D.K + x) * G + blockIdx.x] = (x == 2) ? __longlong_as_double((long long)m) : v;
    }
  }
  if (last_block_2d(counter)) {
    // one warp per output: lanes take a fixed strided share of the blocks,
    // then a butterfly
    const int nout = hist_dots_outputs(D.K);
    for (int o = warp; o < nout; o += kWarps) {
      const bool is_max = (o == nout - 1);
      double v = 0.0;
      unsigned long long m = 0ull;
      for (int bx = lane; bx < G; bx += 32) {
        const double u = partials[(int64_t)o * G + bx];
        if (is_max) m = max(m, (unsigned long long)__double_as_longlong(u));
        else v += u;
      }
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, s);
        m = max(m, __shfl_xor_sync(0xffffffffu, m, s));
      }
      if (lane == 0) out[o] = is_max ? __longlong_as_double((long long)m) : v;
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// out = cg g + sum_k c_k h_k in float64, the terms added in a fixed order.
__global__ void __launch_bounds__(kThreads) hist_comb_kernel(const HistComb C, int64_t n, double* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll 8
    for (int k = 0; k < C.K; k++) s = fma(C.c[k], C.h[k][e], s);
    out[e] = fma(C.cg, C.g[e], s);
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

// At least kPerThread elements per thread: every block ends in butterflies,
// so short vectors get few blocks.
int hist_dots_blocks(int64_t n) {
  int64_t b = (n + (int64_t)kThreads * kPerThread - 1) / ((int64_t)kThreads * kPerThread);
  if (b < 1) b = 1;
  if (b > kMaxDotBlocks) b = kMaxDotBlocks;
  return (int)b;
}

cudaError_t launch_hist_dots(const HistDots& hd, int64_t n, double* partials, unsigned* counter, double* out,
                             cudaStream_t s) {
  if (hd.K < 0 || hd.K > kMaxHist) return cudaErrorInvalidValue;
  const int G = hist_dots_blocks(n);
  const int rows = hd.K > 0 ? (hd.K + kHistChunk - 1) / kHistChunk : 1;
  hist_dots_kernel<<<dim3(G, rows), kThreads, 0, s>>>(hd, n, partials, counter, out);
  return cudaGetLastError();
}

cudaError_t launch_hist_comb(const HistComb& hc, int64_t n, double* out, cudaStream_t s) {
  if (hc.K < 0 || hc.K > kMaxHist) return cudaErrorInvalidValue;
  hist_comb_kernel<<<grid_for(n), kThreads, 0, s>>>(hc, n, out);
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
