// Regulariser, mean term and the final deterministic reductions of one
// objective evaluation (Ploner et al., Eq. 1 and Sec. 2.1).
//
//   msum_kernel: S_c = sum over both volumes and all A-scans of component c
//                (the three sums of the mean term M).
//   reg_kernel:  per A-scan, the temporal regulariser along each volume's
//                acquisition chain (pairs n, n+1 weighted by omega_n,
//                pseudo-Huber of the displacement difference) and its
//                gradient, plus dM/dD = 2 mu S_c, are added to the float
//                data-term gradient and the sum is written as the float64
//                gradient; the partial sums of S^str, S^ang, R and grad . dir
//                are reduced to f = eta S^str + S^ang / eta + alpha R +
//                mu sum_c S_c^2.
//
// Per-element arithmetic is float (double arithmetic is 1/64 of the float
// rate on this GPU, with a long latency) except for the few float64
// operations that fix the precision: displacement differences (formed in
// float64, rounded once), the mean-term sums and the line-search product
// grad . dir.  Each thread's float partials are widened exactly and every sum
// across threads and blocks is a float64 tree with a fixed shape.  The grid is fixed for a given size and the "last block
// finishes" pattern adds the block partials: no waits, no float atomics,
// bitwise reproducible.
#include "common.cuh"
#include "solve.cuh"

namespace octmc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMsumBlocks = 152;
constexpr int kMaxRegBlocks = 608;

// Sum of v[c] over the block, result valid in thread 0 (fixed tree).
template <int N>
__device__ void block_sum(double (&v)[N]) {
  __shared__ double sm[N][kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < N; c++) {
    const double s = warp_sum(v[c]);
    if (lane == 0) sm[c][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < N; c++) {
      double s = lane < kWarps ? sm[c][lane] : 0.0;
#pragma unroll
      for (int o = kWarps / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      v[c] = s;
    }
  }
  __syncthreads();
}

// Maximum of v over the block, valid in thread 0.
__device__ unsigned long long block_max(unsigned long long v) {
  __shared__ unsigned long long sm[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < kWarps; w++) v = max(v, sm[w]);
  __syncthreads();
  return v;
}

// True in every thread of the last of nblk blocks to finish (partials visible).
__device__ bool last_block(unsigned* counter, int nblk) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == (unsigned)nblk - 1u);
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// The last block adds partials[b * N + c] over the blocks b, in a fixed
// strided order per thread followed by block_sum.  Result in thread 0.
template <int N>
__device__ void sum_partials(const double* partials, int nblocks, double (&v)[N]) {
#pragma unroll
  for (int c = 0; c < N; c++) v[c] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
    for (int c = 0; c < N; c++) v[c] += partials[b * N + c];
  block_sum<N>(v);
}

// Block blk of nblk blocks working on one problem's mean-term sums.
__device__ void msum_body(const double* __restrict__ disp, int64_t plane, EvalResult* res, double* partials,
                          unsigned* counter, int blk, int nblk) {
  // float64 throughout: the sums S_c nearly cancel at a centred field, so
  // their relative error is that of the inputs' magnitudes (6 adds per A-scan)
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t e = (int64_t)blk * kThreads + threadIdx.x; e < plane; e += (int64_t)nblk * kThreads) {
#pragma unroll
    for (int c = 0; c < 3; c++) v[c] += disp[c * plane + e] + disp[(3 + c) * plane + e];
  }
  block_sum<3>(v);
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; c++) partials[blk * 3 + c] = v[c];
  if (last_block(counter, nblk)) {
    sum_partials<3>(partials, nblk, v);
    if (threadIdx.x == 0) {
      for (int c = 0; c < 3; c++) res->msum[c] = v[c];
      *counter = 0u;
    }
  }
}

__global__ void __launch_bounds__(kThreads) msum_kernel(const double* __restrict__ disp, int64_t plane,
                                                        EvalResult* res, double* partials,
                                                        unsigned* counter) {
  msum_body(disp, plane, res, partials, counter, blockIdx.x, gridDim.x);
}

// Slot of block b: the last s with b0[s] <= b (block-uniform).
__device__ __forceinline__ int slot_of(const int* b0, int nslots, int b) {
  int lo = 0, hi = nslots - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b0[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads) msum_multi_kernel(const __grid_constant__ MsumMulti M) {
  const int s = slot_of(M.b0, M.nslots, blockIdx.x);
  const MsumSlot& S = M.sl[s];
  msum_body(S.disp, S.plane, S.res, S.partials, S.counter, blockIdx.x - M.b0[s], M.b0[s + 1] - M.b0[s]);
}

// Pseudo-Huber loss (and derivative) of a displacement difference.
__device__ __forceinline__ float huber(float x, float inv_eps, float* dl) {
  const float r = x * inv_eps;
  const float q = fmaf(r, r, 1.0f);
  const float is = rsqrtf(q);
  *dl = r * is;
  return __fdividef(x * r, fmaf(q, is, 1.0f));
}

__device__ void reg_body(const RegArgs& A, int blk, int nblk) {
  const LevelDev& L = A.L;
  const int64_t n = (int64_t)L.w * L.h;
  const float inv_eps = (float)(1.0 / A.eps_r);
  // every pair of the chain carries the level depth d (the per-A-scan scale
  // of the data term, as the angio term of Eq. 6 does)
  const float alpha_d = (float)(A.alpha * (double)L.d);
  float two_mu_s[3];
#pragma unroll
  for (int c = 0; c < 3; c++) two_mu_s[c] = (float)(2.0 * A.mu * A.result->msum[c]);
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // S^str, S^ang, R, grad . dir
  unsigned long long gmx = 0ull;       // max |grad| as the bits of a non-negative float64
  // one work item per A-scan and scan (2 n items): the three components of
  // one volume's displacement; the A-scan's S^str, S^ang go with scan X
  for (int64_t e = (int64_t)blk * kThreads + threadIdx.x; e < 2 * n; e += (int64_t)nblk * kThreads) {
    const int V = e >= n ? 1 : 0;
    const int64_t p = e - V * n;
    float r = 0.f;
    double gd = 0.0;
    const int nx = L.next[V][p], pv = L.prev[V][p];
    const float wn = nx >= 0 ? L.wnext[V][p] : 0.f;
    const float wp = pv >= 0 ? L.wprev[V][p] : 0.f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const double* dc = A.disp + (V * 3 + c) * n;
      const double x = dc[p];
      float gr = 0.f;
      if (nx >= 0) {  // pair (p, next) is counted at its first sample
        float dl;
        r = fmaf(wn, huber((float)(dc[nx] - x), inv_eps, &dl), r);  // float64 difference, rounded once
        gr = fmaf(-wn, dl, gr);
      }
      if (pv >= 0) {
        float dl;
        huber((float)(x - dc[pv]), inv_eps, &dl);
        gr = fmaf(wp, dl, gr);
      }
      if (A.grad) {
        const int64_t gi = (V * 3 + c) * n + p;
        const float g = A.gdata[gi] + fmaf(alpha_d, gr, two_mu_s[c]);
        const double gw = widen_exact(g);
        A.grad[gi] = gw;
        if (A.dir) gd = fma(gw, A.dir[gi], gd);  // line-search product in float64
        gmx = max(gmx, (unsigned long long)__double_as_longlong(gw) & 0x7fffffffffffffffull);
      }
    }
    if (V == 0) {
      v[0] += widen_exact(A.str_in[p]);
      v[1] += widen_exact(A.ang_in[p]);
    }
    v[2] += widen_exact(r);
    v[3] += gd;
  }
  block_sum<4>(v);
  gmx = block_max(gmx);
  if (threadIdx.x == 0) {
    for (int c = 0; c < 4; c++) A.partials[blk * 4 + c] = v[c];
    A.partials[4 * nblk + blk] = __longlong_as_double((long long)gmx);
  }
  if (last_block(A.counter, nblk)) {
    sum_partials<4>(A.partials, nblk, v);
    unsigned long long m = 0ull;
    for (int b = threadIdx.x; b < nblk; b += kThreads)
      m = max(m, (unsigned long long)__double_as_longlong(A.partials[4 * nblk + b]));
    m = block_max(m);
    if (threadIdx.x == 0) {
      const double* ms = A.result->msum;
      const double M = A.mu * (ms[0] * ms[0] + ms[1] * ms[1] + ms[2] * ms[2]);
      EvalResult* res = A.result;
      res->terms[0] = v[0];
      res->terms[1] = v[1];
      const double eta = A.eta_dev ? *A.eta_dev : A.eta;
      const double R = (double)L.d * v[2];
      res->terms[2] = R;
      res->terms[3] = M;
      res->terms[4] = eta * v[0] + v[1] / eta + A.alpha * R + M;
      res->terms[5] = eta;
      res->gdir = v[3];
      *A.counter = 0u;
      if (A.ctl) ls_decide(A.ctl, res->terms[4], v[3], __longlong_as_double((long long)m), A.h_branch, A.h_while);
    }
  }
}

__global__ void __launch_bounds__(kThreads) reg_kernel(const RegArgs A) { reg_body(A, blockIdx.x, gridDim.x); }

__global__ void __launch_bounds__(kThreads) reg_multi_kernel(const __grid_constant__ RegMulti M) {
  const int s = slot_of(M.b0, M.nslots, blockIdx.x);
  reg_body(M.ra[s], blockIdx.x - M.b0[s], M.b0[s + 1] - M.b0[s]);
}

}  // namespace

int msum_grid_blocks() { return kMsumBlocks; }

cudaError_t launch_msum_multi(const MsumMulti& M, cudaStream_t s) {
  if (M.nslots <= 0 || M.b0[M.nslots] <= 0) return cudaSuccess;
  msum_multi_kernel<<<M.b0[M.nslots], kThreads, 0, s>>>(M);
  return cudaGetLastError();
}

cudaError_t launch_reg_multi(const RegMulti& M, cudaStream_t s) {
  if (M.nslots <= 0 || M.b0[M.nslots] <= 0) return cudaSuccess;
  reg_multi_kernel<<<M.b0[M.nslots], kThreads, 0, s>>>(M);
  return cudaGetLastError();
}

int reg_grid_blocks(int64_t n) {
  int64_t b = (2 * n + kThreads - 1) / kThreads;
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
