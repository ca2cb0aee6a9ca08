// Regulariser, mean term and the final deterministic reductions of one
// objective evaluation (Ploner et al., Eq. 1 and Sec. 2.1).
//
//   msum_kernel: S_c = sum over both volumes and all A-scans of component c
//                (the three sums of the mean term M).
//   reg_kernel:  per A-scan, the temporal regulariser along each volume's
//                acquisition chain (pairs n, n+1 weighted by omega_n,
//                pseudo-Huber of the displacement difference), its gradient
//                and dM/dD = 2 mu S_c are added to the data gradient; the
//                block partial sums of S^str, S^ang, R and grad . dir are
//                reduced by the last block in a fixed order:
//                f = eta S^str + S^ang / eta + alpha R + mu sum_c S_c^2.
// Both use a fixed grid and the "last block finishes" pattern: every block
// writes its partials, the block that increments the counter last adds the
// partials in block order and resets the counter.  No waits, no float
// atomics, bitwise reproducible.
#include "common.cuh"

namespace octmc {
namespace {

constexpr int kThreads = 256;
constexpr int kMsumBlocks = 304;   // 2 x 152 SMs
constexpr int kMaxRegBlocks = 1216;

template <int N>
__device__ void block_sum(double (&v)[N], double* smem /* [N][kThreads/32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < N; c++) {
    double s = warp_sum(v[c]);
    if (lane == 0) smem[c * (kThreads / 32) + warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < N; c++) {
      double s = 0.0;
      for (int w = 0; w < kThreads / 32; w++) s += smem[c * (kThreads / 32) + w];
      v[c] = s;
    }
  }
}

// Returns true in thread 0 of the last block to finish (partials visible).
__device__ bool last_block(unsigned* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    return true;
  }
  return false;
}

__global__ void __launch_bounds__(kThreads) msum_kernel(const double* __restrict__ disp, int64_t plane,
                                                        EvalResult* res, double* partials,
                                                        unsigned* counter) {
  __shared__ double sm[3 * (kThreads / 32)];
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < plane;
       e += (int64_t)gridDim.x * kThreads) {
#pragma unroll
    for (int c = 0; c < 3; c++) v[c] += disp[c * plane + e] + disp[(3 + c) * plane + e];
  }
  block_sum<3>(v, sm);
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; c++) partials[blockIdx.x * 3 + c] = v[c];
  if (last_block(counter)) {
    for (int c = 0; c < 3; c++) {
      double s = 0.0;
      for (unsigned b = 0; b < gridDim.x; b++) s += partials[b * 3 + c];
      res->msum[c] = s;
    }
    *counter = 0u;
  }
}

// Pseudo-Huber loss of a displacement difference (float: the differences
// are O(1) px and the sums are taken in double).
__device__ __forceinline__ float huber(float x, float inv_eps, float* dl) {
  const float r = x * inv_eps;
  const float q = fmaf(r, r, 1.0f);
  const float is = rsqrtf(q);
  *dl = r * is;
  return __fdividef(x * r, fmaf(q, is, 1.0f));
}

__global__ void __launch_bounds__(kThreads) reg_kernel(const RegArgs A) {
  __shared__ double sm[4 * (kThreads / 32)];
  const LevelDev& L = A.L;
  const int64_t n = (int64_t)L.w * L.h;
  const float inv_eps = (float)(1.0 / A.eps_r);
  const double two_mu_s[3] = {2.0 * A.mu * A.result->msum[0], 2.0 * A.mu * A.result->msum[1],
                              2.0 * A.mu * A.result->msum[2]};
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // S^str, S^ang, R, grad . dir
  for (int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * kThreads) {
    v[0] += A.str_in[p];
    v[1] += A.ang_in[p];
#pragma unroll
    for (int V = 0; V < 2; V++) {
      const int nx = L.next[V][p], pv = L.prev[V][p];
      const double wn = nx >= 0 ? L.wnext[V][p] : 0.0;
      const double wp = pv >= 0 ? L.wprev[V][p] : 0.0;
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const double* dc = A.disp + (V * 3 + c) * n;
        const double x = dc[p];
        double gr = 0.0;
        if (nx >= 0) {  // pair (p, next) is counted at its first sample
          float dl;
          const float lv = huber((float)(dc[nx] - x), inv_eps, &dl);
          v[2] += wn * (double)lv;
          gr -= wn * (double)dl;
        }
        if (pv >= 0) {
          float dl;
          huber((float)(x - dc[pv]), inv_eps, &dl);
          gr += wp * (double)dl;
        }
        if (A.grad) {
          const int64_t gi = (V * 3 + c) * n + p;
          const double g = A.grad[gi] + A.alpha * gr + two_mu_s[c];
          A.grad[gi] = g;
          if (A.dir) v[3] += g * A.dir[gi];
        }
      }
    }
  }
  block_sum<4>(v, sm);
  if (threadIdx.x == 0)
    for (int c = 0; c < 4; c++) A.partials[blockIdx.x * 4 + c] = v[c];
  if (last_block(A.counter)) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned b = 0; b < gridDim.x; b++)
      for (int c = 0; c < 4; c++) s[c] += A.partials[b * 4 + c];
    const double* ms = A.result->msum;
    const double M = A.mu * (ms[0] * ms[0] + ms[1] * ms[1] + ms[2] * ms[2]);
    EvalResult* r = A.result;
    r->terms[0] = s[0];
    r->terms[1] = s[1];
    r->terms[2] = s[2];
    r->terms[3] = M;
    r->terms[4] = A.eta * s[0] + s[1] / A.eta + A.alpha * s[2] + M;
    r->terms[5] = A.eta;
    r->gdir = s[3];
    *A.counter = 0u;
  }
}

}  // namespace

int msum_grid_blocks() { return kMsumBlocks; }

int reg_grid_blocks(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  return (int)(b < 1 ? 1 : (b > kMaxRegBlocks ? kMaxRegBlocks : b));
}

cudaError_t launch_msum(const double* disp, int64_t plane, EvalResult* res, double* partials,
                        unsigned* counter, cudaStream_t s) {
  msum_kernel<<<kMsumBlocks, kThreads, 0, s>>>(disp, plane, res, partials, counter);
  return cudaGetLastError();
}

cudaError_t launch_reg(const RegArgs& a, cudaStream_t s) {
  const int blocks = reg_grid_blocks((int64_t)a.L.w * a.L.h);
  reg_kernel<<<blocks, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace octmc
