// Persistent small-level solve (Ploner et al., Sec. 2.1: L-BFGS in a factor-2
// multi-resolution pyramid).  On the coarse levels one evaluation is a few
// microseconds of arithmetic spread over a handful of kernels, so launch and
// tail latency dominate.  Here one cooperative kernel -- one block of 1024
// threads per SM -- runs the whole loop of a level:
//
//   P1  trial point: after a new iterate x <- xs, g <- gs; after new
//       coefficients dir = cg g + sum_j coef_j h_j; the save of the best
//       Armijo point; xt = x + a dir; block partials of the mean-term sums
//   --- grid barrier
//   P2  evaluation at xt: the data term of each A-scan by one warp, then in
//       the same warp its regulariser terms, mean-term gradient and float64
//       gradient (Eq. 1-10); block partials of S^str, S^ang, R, grad . dir,
//       max |grad|
//   --- grid barrier
//   P3  every block adds the partials (same order everywhere) and takes the
//       line-search decision and stopping tests on its own shared-memory copy
//       of the state: all blocks take the same decision without exchanging it
//   P4  after a new iterate or a retry: the new pair and the history
//       products, block partials
//   --- grid barrier
//   P5  every block adds the products' partials and runs the history update
//       and the compact-form algebra on its copy of the state
//
// The operations are those of the kernels of the graph-driven loop (the same
// objective, gradient, decision and algebra), with other reduction orders.
// Every grid barrier waits with an iteration cap and a %globaltimer limit;
// when one runs out the kernel records it (status 3) and every block leaves
// the loop.
#include <math.h>

#include "common.cuh"
#include "data.cuh"
#include "reg_ascan.cuh"
#include "solve.cuh"
#include "solve_algebra.cuh"

namespace octmc {
namespace {

constexpr int kLThreads = 1024;
constexpr int kLWarps = kLThreads / 32;
constexpr int kMaxVec = 2 * kMaxM + 2;
constexpr int kP4 = 2 * (2 * kMaxM + 2) + 2;  // products per block: 2 per candidate + y.y + g.g
constexpr int kPartStride = 3 + 5 + kP4;      // doubles per block of scratch
constexpr unsigned long long kBarrierNs = 2000000000ull;  // 2 s
constexpr unsigned long long kBarrierSpins = 1ull << 25;

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (every block resident).  bar[0]
// counts arrivals, bar[1] is the generation; the last block to arrive resets
// the count and opens the next generation.  A waiting block gives up after
// kBarrierSpins polls or kBarrierNs and sets *err; every waiting block also
// leaves once *err is set.  Returns false (in every thread) once *err is set.
__device__ bool grid_barrier(unsigned* bar, int* err, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    volatile int* verr = err;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1u) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = now_ns();
      unsigned long long spins = 0;
      while (*gen == g0) {
        if (*verr) break;
        if (++spins > kBarrierSpins || now_ns() - t0 > kBarrierNs) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = (*verr == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// Block sum of N doubles per thread, result in thread 0 (fixed tree).
template <int N>
__device__ void lblock_sum(double (&v)[N]) {
  __shared__ double sm[N][kLWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < N; c++) {
    const double t = warp_sum(v[c]);
    if (lane == 0) sm[c][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < N; c++) {
      double t = 0.0;
      for (int w = 0; w < kLWarps; w++) t += sm[c][w];
      v[c] = t;
    }
  }
  __syncthreads();
}

// Block maximum of non-negative float64 bit patterns, result in thread 0.
__device__ unsigned long long lblock_max(unsigned long long v) {
  __shared__ unsigned long long sm[kLWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 0; w < kLWarps; w++) v = max(v, sm[w]);
  __syncthreads();
  return v;
}

__device__ __forceinline__ const double* lhvec(const HistSet& H, int id) {
  return (id & 1) ? H.Y[id >> 1] : H.S[id >> 1];
}

template <typename T>
__global__ void __launch_bounds__(kLThreads, 1) level_kernel(const __grid_constant__ LevelArgs A) {
  __shared__ SolveState sS;
  __shared__ Algebra alg;
  __shared__ double s_ms[3];
  __shared__ double s_tot[4];
  __shared__ unsigned long long s_gmax;
  __shared__ const double* s_hp[kMaxVec];
  __shared__ double s_cf[kMaxVec];
  copy_state<kLThreads>(&sS, A.S);
  __syncthreads();
  const int G = gridDim.x, B = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SolveVecs& V = A.V;
  const LevelDev& L = A.D.L;
  const int64_t plane = V.plane, n = V.n;
  double* const part1 = A.part;                       // [G][3] mean-term sums
  double* const part2 = A.part + (int64_t)3 * G;      // [G][5] S^str, S^ang, R, grad . dir, max |grad|
  double* const part4 = A.part + (int64_t)8 * G;      // [G][kP4] products
  const float inv_eps_r = (float)(1.0 / A.eps_r);
  const float alpha_d = (float)(A.alpha * (double)L.d);
  bool ok = true;
  for (;;) {
    // ---- P1: the trial point (the n = 6 plane elements spread over the grid)
    {
      const bool init = sS.mode == kModeInit;
      const bool branch = sS.branch != 0;
      const bool moved = sS.moved != 0;
      const bool save = sS.save_best && !branch;
      const bool best = sS.restore_best && !sS.save_best;
      const double* xs = best ? V.xb : V.xt;
      const double* gs = best ? V.gb : V.gt;
      const double a = sS.a, cg = sS.cg;
      const int nc = branch ? sS.nc : 0;
      if (tid < nc) {
        s_hp[tid] = lhvec(A.H, sS.hid[tid]);
        s_cf[tid] = sS.coef[tid];
      }
      __syncthreads();
      double ms[3] = {0.0, 0.0, 0.0};
      for (int64_t e = (int64_t)B * kLThreads + tid; e < n; e += (int64_t)G * kLThreads) {
        double xe, ge = 0.0;
        if (moved) {
          xe = xs[e];
          ge = gs[e];
          V.x[e] = xe;
          V.g[e] = ge;
        } else {
          xe = V.x[e];
          if (branch) ge = V.g[e];
        }
        if (save) {
          V.xb[e] = V.xt[e];
          V.gb[e] = V.gt[e];
        }
        double d;
        if (branch) {
          double t0 = 0.0, t1 = 0.0;
          int j = 0;
          for (; j + 1 < nc; j += 2) {
            t0 = fma(s_cf[j], __ldg(s_hp[j] + e), t0);
            t1 = fma(s_cf[j + 1], __ldg(s_hp[j + 1] + e), t1);
          }
          if (j < nc) t0 = fma(s_cf[j], __ldg(s_hp[j] + e), t0);
          d = fma(cg, ge, t0 + t1);
          V.dir[e] = d;
        } else {
          d = V.dir[e];
        }
        const double xn = init ? xe : fma(a, d, xe);
        V.xt[e] = xn;
        const int comp = (int)((uint64_t)e / (uint64_t)plane) % 3;
        ms[0] += comp == 0 ? xn : 0.0;
        ms[1] += comp == 1 ? xn : 0.0;
        ms[2] += comp == 2 ? xn : 0.0;
      }
      lblock_sum<3>(ms);
      if (tid == 0)
        for (int c = 0; c < 3; c++) part1[B * 3 + c] = ms[c];
    }
    ok = grid_barrier(A.bar, A.err, G);
    if (!ok) break;
    // ---- P2: the evaluation at xt
    {
      if (warp == 0) {  // the mean-term sums S_c (same order in every block)
        for (int c = 0; c < 3; c++) {
          double t = 0.0;
          for (int b = lane; b < G; b += 32) t += part1[b * 3 + c];
          t = warp_sum(t);
          if (lane == 0) s_ms[c] = t;
        }
      }
      __syncthreads();
      double acc[4] = {0.0, 0.0, 0.0, 0.0};  // S^str, S^ang, R, grad . dir
      unsigned long long gmx = 0ull;
      const float two_mu_s = (float)(2.0 * A.mu * s_ms[lane < 6 ? lane % 3 : 0]);
      for (int64_t p = (int64_t)B * kLWarps + warp; p < plane; p += (int64_t)G * kLWarps)
        eval_ascan<T>(A.D, V.gt, V.dir, p, lane, two_mu_s, inv_eps_r, alpha_d, acc, &gmx);
      lblock_sum<4>(acc);
      gmx = lblock_max(gmx);
      if (tid == 0) {
        for (int c = 0; c < 4; c++) part2[B * 5 + c] = acc[c];
        part2[B * 5 + 4] = __longlong_as_double((long long)gmx);
      }
    }
    ok = grid_barrier(A.bar, A.err, G);
    if (!ok) break;
    // ---- P3: the line-search decision, taken by every block on its copy
    {
      if (warp == 0) {
        for (int c = 0; c < 4; c++) {
          double t = 0.0;
          for (int b = lane; b < G; b += 32) t += part2[b * 5 + c];
          t = warp_sum(t);
          if (lane == 0) s_tot[c] = t;
        }
        unsigned long long m = 0ull;
        for (int b = lane; b < G; b += 32) m = max(m, (unsigned long long)__double_as_longlong(part2[b * 5 + 4]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_gmax = m;
      }
      __syncthreads();
      if (tid == 0) {
        const double M = A.mu * (s_ms[0] * s_ms[0] + s_ms[1] * s_ms[1] + s_ms[2] * s_ms[2]);
        const double eta = sS.eta;
        const double R = (double)L.d * s_tot[2];
        const double f = eta * s_tot[0] + s_tot[1] / eta + A.alpha * R + M;
        ls_decide_state(&sS, f, s_tot[3], __longlong_as_double((long long)s_gmax));
      }
      __syncthreads();
      if (!ls_more(&sS)) break;
      if (!sS.branch) continue;
    }
    // ---- P4: the new pair and the history products.  The block's
    // contiguous share of the elements; warp w takes candidates w, w + 32, ...
    // (and, as candidate K, y . y and g . g); the new pair is formed from xs,
    // x, gp, g by the warps of its two slots, which store it
    const int mode = sS.mode;
    const bool accepted = mode == kModeAccept;
    const int nstored = sS.k;
    const int ncand = nstored + (accepted ? 1 : 0);
    const int K = 2 * ncand;
    {
      const bool best = sS.restore_best && !sS.save_best;
      const double* xs = best ? V.xb : V.xt;
      const double* gp = (mode == kModeRetry) ? V.g : (best ? V.gb : V.gt);
      double* sv = A.H.S[sS.spare];
      double* yv = A.H.Y[sS.spare];
      const int64_t share = ((n + G - 1) / G + 31) / 32 * 32;
      const int64_t e0 = min(n, (int64_t)B * share), e1 = min(n, e0 + share);
      for (int c = warp; c <= K; c += kLWarps) {
        double a0 = 0.0, a1 = 0.0;
        if (c < K) {
          const int t = c >> 1;
          const bool is_new = accepted && t == nstored;
          const double* hc = is_new ? nullptr : ((c & 1) ? A.H.Y[sS.order[t]] : A.H.S[sS.order[t]]);
          for (int64_t e = e0 + lane; e < e1; e += 32) {
            const double gv = __ldg(gp + e);
            const double yn = accepted ? gv - __ldg(V.g + e) : 0.0;
            double hv;
            if (is_new) {
              if (c & 1) {
                hv = yn;
                yv[e] = hv;
              } else {
                hv = __ldg(xs + e) - __ldg(V.x + e);
                sv[e] = hv;
              }
            } else {
              hv = __ldg(hc + e);
            }
            if (accepted) a0 = fma(hv, yn, a0);
            a1 = fma(hv, gv, a1);
          }
        } else {
          for (int64_t e = e0 + lane; e < e1; e += 32) {
            const double gv = __ldg(gp + e);
            if (accepted) {
              const double yn = gv - __ldg(V.g + e);
              a0 = fma(yn, yn, a0);
            }
            a1 = fma(gv, gv, a1);
          }
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        if (lane == 0) {
          part4[(int64_t)B * kP4 + 2 * c] = a0;
          part4[(int64_t)B * kP4 + 2 * c + 1] = a1;
        }
      }
    }
    ok = grid_barrier(A.bar, A.err, G);
    if (!ok) break;
    // ---- P5: the products' totals, the history update and the algebra
    {
      // outputs: [2v] = h_v . y, [2v+1] = h_v . g, [2K] = y . y, [2K+1] = g . g
      for (int o = warp; o < 2 * K + 2; o += kLWarps) {
        double t = 0.0;
        for (int b = lane; b < G; b += 32) t += part4[(int64_t)b * kP4 + o];
        t = warp_sum(t);
        if (lane == 0) sS.dots[o] = t;
      }
      __syncthreads();
      if (tid == 0) {
        sS.ncand = ncand;
        for (int t = 0; t < ncand; t++) sS.cand[t] = (t < nstored) ? sS.order[t] : sS.spare;
      }
      __syncthreads();
      after_products(&sS, alg);
      __syncthreads();
    }
  }
  // ---- the end of the level: the last new iterate becomes x; block 0
  // writes the state back (status 3 when a grid barrier timed out)
  if (!ok) {
    if (tid == 0) {
      sS.status = 3;
      sS.done = 1;
    }
  } else if (sS.moved) {
    const bool best = sS.restore_best && !sS.save_best;
    const double* xs = best ? V.xb : V.xt;
    for (int64_t e = (int64_t)B * kLThreads + tid; e < n; e += (int64_t)G * kLThreads) V.x[e] = xs[e];
  }
  __syncthreads();
  if (B == 0) copy_state<kLThreads>(A.S, &sS);
}

// One grid barrier that waits for `extra` more blocks than the grid has:
// with extra > 0 no block can complete it, so every wait runs out (bounded
// as in the level kernel) and sets *err.  Tests the bounded wait.
__global__ void __launch_bounds__(kLThreads, 1) barrier_probe_kernel(unsigned* bar, int* err, int extra) {
  grid_barrier(bar, err, gridDim.x + (unsigned)extra);
}

template <typename T>
int level_grid_for() {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, level_kernel<T>, kLThreads, 0) != cudaSuccess)
    return 0;
  return per_sm >= 1 ? device_sm_count() : 0;  // one block per SM
}

template <typename T>
cudaError_t launch_level_t(const LevelArgs& A, cudaStream_t s) {
  const int grid = level_grid_for<T>();
  if (grid < 1) return cudaErrorCooperativeLaunchTooLarge;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kLThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, level_kernel<T>, A);
}

}  // namespace

int level_grid(int dtype) {
  if (dtype == OCTMC_BF16) return level_grid_for<__nv_bfloat16>();
  if (dtype == OCTMC_F16) return level_grid_for<__half>();
  return level_grid_for<float>();
}

int64_t level_part_doubles(int grid) { return (int64_t)grid * kPartStride; }

cudaError_t launch_barrier_probe(unsigned* bar, int* err, int extra, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_probe_kernel, kLThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)device_sm_count());
  cfg.blockDim = dim3(kLThreads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, barrier_probe_kernel, bar, err, extra);
}

cudaError_t launch_level_persistent(const LevelArgs& A, int dtype, cudaStream_t s) {
  if (dtype == OCTMC_BF16) return launch_level_t<__nv_bfloat16>(A, s);
  if (dtype == OCTMC_F16) return launch_level_t<__half>(A, s);
  return launch_level_t<float>(A, s);
}

}  // namespace octmc
