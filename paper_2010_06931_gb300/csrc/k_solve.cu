// Kernels of the device-resident level solve (Ploner et al., Sec. 2.1:
// "gradient-based L-BFGS solver").  One loop iteration is four kernels: the
// trial kernel (the direction and the iterate left by the last decision, the
// trial point, the mean-term sums), the data and regulariser kernels of the
// evaluation (the regulariser's last block takes the line-search decision
// and the stopping tests), and, after a new iterate or a retry, the products
// kernel (history pair, history products, compact-form (Byrd, Nocedal &
// Schnabel) direction coefficients).  All state lives in one SolveState in
// device memory; the host launches one graph per solve and reads the state
// once at the end.
//
// The products and the small dense algebra are float64 with fixed
// reduction trees and a fixed operation order, so a solve is reproducible
// bit for bit.
#include <math.h>

#include "common.cuh"
#include "solve_algebra.cuh"

namespace octmc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 20;             // history vectors per block row
constexpr int kMaxVec = 2 * kMaxM + 2; // history vectors of one product pass
constexpr int kVals = 64;              // per-thread partial sums of the products (2 kChunk + 2, padded)

__device__ __forceinline__ const double* hvec(const HistSet& H, int id) {
  return (id & 1) ? H.Y[id >> 1] : H.S[id >> 1];
}

// Sum of v over the block, valid in thread 0 (fixed tree).
__device__ double block_sum1(double v) {
  __shared__ double sm[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    v = 0.0;
    for (int w = 0; w < kWarps; w++) v += sm[w];
  }
  __syncthreads();
  return v;
}

// One trial point of the line search, after what the last decision left to
// do (Sec. 2.1):
//  - a new iterate (the start point or an accepted step): x <- xs, g <- gs,
//    xs being the last trial, or the saved best Armijo point when the search
//    ended on it (unless that point is the last trial itself);
//  - the previous trial kept as the best Armijo point while the search goes
//    on: saved to xb, gb before xt is overwritten (gt is overwritten by the
//    evaluation that follows);
//  - new direction coefficients (after a new iterate or a retry): dir = cg g +
//    sum_j coef_j h_j (float64, even and odd terms summed separately, in a
//    fixed order);
//  - xt = x + a dir (x itself for the level's start evaluation);
//  - the mean-term sums S_c of xt over both scans (Eq. 1, M; float64, fixed
//    trees), reduced by the last block into res->msum.
// Grid (Gx, 6): blockIdx.y is the displacement plane (scan V, component c:
// plane 3 V + c), so every block has one plane's share and enough blocks
// run to hide the float64 latency of the direction sums.
__global__ void __launch_bounds__(kThreads) trial_kernel(const SolveState* __restrict__ S, const HistSet H,
                                                         const SolveVecs V, EvalResult* res, double* partials,
                                                         unsigned* counter) {
  __shared__ const double* hp[kMaxVec];
  __shared__ double cf[kMaxVec];
  __shared__ bool is_last;
  const bool init = S->mode == kModeInit;
  const bool branch = S->branch != 0;
  const bool moved = S->moved != 0;
  const bool save = S->save_best && !branch;
  const bool best = S->restore_best && !S->save_best;
  const double* xs = best ? V.xb : V.xt;
  const double* gs = best ? V.gb : V.gt;
  const double a = S->a, cg = S->cg;
  const int nc = branch ? S->nc : 0;
  if (threadIdx.x < nc) {
    hp[threadIdx.x] = hvec(H, S->hid[threadIdx.x]);
    cf[threadIdx.x] = S->coef[threadIdx.x];
  }
  __syncthreads();
  const int Gx = gridDim.x, k = blockIdx.y;
  const int64_t plane = V.plane;
  double ms = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x; p < plane; p += (int64_t)Gx * kThreads) {
    const int64_t e = k * plane + p;
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
      // two interleaved chains (even / odd terms, fixed order) halve the
      // dependent float64 latency; the history is read-only here
      double t0 = 0.0, t1 = 0.0;
      int j = 0;
      for (; j + 1 < nc; j += 2) {
        t0 = fma(cf[j], __ldg(hp[j] + e), t0);
        t1 = fma(cf[j + 1], __ldg(hp[j + 1] + e), t1);
      }
      if (j < nc) t0 = fma(cf[j], __ldg(hp[j] + e), t0);
      d = fma(cg, ge, t0 + t1);
      V.dir[e] = d;
    } else {
      d = V.dir[e];
    }
    const double xn = init ? xe : fma(a, d, xe);
    V.xt[e] = xn;
    ms += xn;
  }
  ms = block_sum1(ms);
  if (threadIdx.x == 0) partials[k * Gx + blockIdx.x] = ms;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == 6u * Gx - 1u);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // S_c: planes c and 3 + c, each over its Gx block partials (fixed order)
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int c = 0; c < 3; c++) {
      double t = 0.0;
      for (int b = lane; b < Gx; b += 32) t += partials[c * Gx + b] + partials[(3 + c) * Gx + b];
      t = warp_sum(t);
      if (lane == 0) res->msum[c] = t;
    }
    if (lane == 0) *counter = 0u;
  }
}

// After the level's loop: the last new iterate (see trial_kernel) becomes x.
__global__ void __launch_bounds__(kThreads) finish_kernel(const SolveState* __restrict__ S, const SolveVecs V) {
  if (!S->moved) return;
  const bool best = S->restore_best && !S->save_best;
  const double* xs = best ? V.xb : V.xt;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < V.n; e += (int64_t)gridDim.x * kThreads)
    V.x[e] = xs[e];
}

// Reduce-scatter of 32 per-lane float64 values over the warp: on return v[0]
// of lane i is the warp total of value i.  Each stage keeps half of the
// values and adds the partner lane's copy of that half, so a lane does 31
// float64 adds for 32 values (a butterfly per value would do 160, and this
// GPU runs float64 at 1/64 of the float rate).  The pairing is fixed, so the
// sums are reproducible.
template <int N>
__device__ __forceinline__ void rs_stage(double* v, int lane) {
  const bool up = (lane & N) != 0;
#pragma unroll
  for (int j = 0; j < N; j++) {
    const double send = up ? v[j] : v[j + N];
    const double keep = up ? v[j + N] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, N);
  }
}

__device__ __forceinline__ double warp_reduce_scatter32(double* v, int lane) {
  rs_stage<16>(v, lane);
  rs_stage<8>(v, lane);
  rs_stage<4>(v, lane);
  rs_stage<2>(v, lane);
  rs_stage<1>(v, lane);
  return v[0];
}

// The products pass over this block's share of the elements, with gp the
// gradient at the iterate the products are for.  After an accepted step the
// new pair s = xs - x, y = gp - g is formed here; the row whose candidates
// include it (slots cs, cs + 1) takes them from registers and stores them.
// v[2c] += h_c . y (accepted step only), v[2c+1] += h_c . gp; first row:
// v[2 kChunk] += y . y, v[2 kChunk + 1] += gp . gp.
template <bool kAccepted>
__device__ __forceinline__ void dots_pass(const double* const* h, int kn, int cs, bool first, bool store,
                                          const double* __restrict__ xs, const double* __restrict__ gp,
                                          const double* __restrict__ x, const double* __restrict__ g,
                                          double* __restrict__ sv, double* __restrict__ yv, int64_t e0, int64_t e1,
                                          double* v) {
  // Every load here is non-coherent (read-only path): none of these vectors
  // is written by this kernel except the spare pair buffers, whose loaded
  // values are discarded for the register copies, so the compiler may batch
  // the loads of later elements ahead of this element's stores.
  for (int64_t e = e0 + threadIdx.x; e < e1; e += kThreads) {
    const double gv = __ldg(gp + e);
    double sn = 0.0, yn = 0.0;
    if (kAccepted) {
      sn = __ldg(xs + e) - __ldg(x + e);
      yn = gv - __ldg(g + e);
    }
#pragma unroll
    for (int c = 0; c < kChunk; c++) {
      if (c < kn) {
        double hv = __ldg(h[c] + e);
        if (kAccepted) hv = (c == cs) ? sn : ((c == cs + 1) ? yn : hv);
        if (kAccepted) v[2 * c] = fma(hv, yn, v[2 * c]);
        v[2 * c + 1] = fma(hv, gv, v[2 * c + 1]);
      }
    }
    if (first) {
      if (kAccepted) v[2 * kChunk] = fma(yn, yn, v[2 * kChunk]);
      v[2 * kChunk + 1] = fma(gv, gv, v[2 * kChunk + 1]);
    }
    if (kAccepted && store) {
      sv[e] = sn;
      yv[e] = yn;
    }
  }
}

// Products of the candidate history vectors (the stored pairs and, after an
// accepted step, the new one) with the probes y_new (accepted step only) and
// the gradient; g . g.  Grid (G, rows): G blocks (one per SM) split the
// elements into contiguous shares, rows cover the problem's longest history
// (block (bx, r) takes candidates r*20 .. r*20+19; rows beyond this step's
// candidates only arrive).  Within a block the float64 partial sums go
// through the reduce-scatter above and a fixed sum over the warps; the last
// block to finish adds the block partials (fixed order) and runs the algebra.
__global__ void __launch_bounds__(kThreads, 1) dots_kernel(SolveState* S, const HistSet H, const SolveVecs V,
                                                           double* partials, unsigned* counter) {
  __shared__ double sm[kVals * kWarps];
  __shared__ bool is_last;
  const int G = gridDim.x;
  const int64_t n = V.n;
  const int mode = S->mode;
  const bool accepted = mode == kModeAccept;
  const int nstored = S->k;
  const int ncand = nstored + (accepted ? 1 : 0);
  const int K = 2 * ncand;
  const int k0 = blockIdx.y * kChunk;
  const int kn = min(kChunk, K - k0);
  const bool first = blockIdx.y == 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (kn <= 0 && !first) {  // a row beyond this step's vectors: only arrive
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1);
    __syncthreads();
    if (!is_last) return;
  } else {
  const double* h[kChunk];
#pragma unroll
  for (int c = 0; c < kChunk; c++) {
    h[c] = nullptr;
    const int v = k0 + c;
    if (c < kn) {
      const int t = v >> 1;
      const int buf = (t < nstored) ? S->order[t] : S->spare;
      h[c] = (v & 1) ? H.Y[buf] : H.S[buf];
    }
  }
  // contiguous share of the elements, a multiple of 32 long (coalesced)
  const int64_t share = ((n + G - 1) / G + 31) / 32 * 32;
  const int64_t e0 = min(n, (int64_t)blockIdx.x * share), e1 = min(n, e0 + share);
  double v[kVals];
#pragma unroll
  for (int c = 0; c < kVals; c++) v[c] = 0.0;
  // the iterate the products are for: the new one (the last trial, or the
  // saved best point), or the current one after a retry
  const bool best = S->restore_best && !S->save_best;
  const double* xs = best ? V.xb : V.xt;
  const double* gp = (mode == kModeRetry) ? V.g : (best ? V.gb : V.gt);
  if (accepted) {
    const int cs = 2 * nstored - k0;  // the new pair's slots in this row (even: both or neither)
    const bool store = cs >= 0 && cs < kn;  // the one row holding them stores the pair
    dots_pass<true>(h, kn, cs, first, store, xs, gp, V.x, V.g, H.S[S->spare], H.Y[S->spare], e0, e1, v);
  } else {
    dots_pass<false>(h, kn, -1, first, false, nullptr, gp, nullptr, nullptr, nullptr, nullptr, e0, e1, v);
  }
  // warp totals: lane i holds values i and 32 + i
  const double t0 = warp_reduce_scatter32(v, lane);
  const double t1 = warp_reduce_scatter32(v + 32, lane);
  sm[lane * kWarps + warp] = t0;
  sm[(32 + lane) * kWarps + warp] = t1;
  __syncthreads();
  // block partials, outputs: [2v] = h_v . y, [2v+1] = h_v . g, [2K] = y . y, [2K+1] = g . g
  const int t = threadIdx.x;
  int out = -1;
  if (t < 2 * kn) out = 2 * k0 + t;
  else if (first && t == 2 * kChunk) out = 2 * K;
  else if (first && t == 2 * kChunk + 1) out = 2 * K + 1;
  if (out >= 0) {
    double a = 0.0;
    for (int w = 0; w < kWarps; w++) a += sm[t * kWarps + w];
    partials[(int64_t)out * G + blockIdx.x] = a;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1);
  __syncthreads();
  if (!is_last) return;
  }
  __threadfence();
  // the epilogue works on a shared-memory copy of the state: its serial parts
  // would otherwise wait on L2 for every dependent access
  __shared__ SolveState sS;
  copy_state<kThreads>(&sS, S);
  __syncthreads();
  const int nout = 2 * K + 2;
  for (int o = warp; o < nout; o += kWarps) {
    double a = 0.0;
    for (int bx = lane; bx < G; bx += 32) a += partials[(int64_t)o * G + bx];
    a = warp_sum(a);
    if (lane == 0) sS.dots[o] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *counter = 0u;
    sS.ncand = ncand;
    for (int c = 0; c < ncand; c++) sS.cand[c] = (c < nstored) ? sS.order[c] : sS.spare;
  }
  __syncthreads();
  __shared__ Algebra alg;
  after_products(&sS, alg);
  __syncthreads();
  copy_state<kThreads>(S, &sS);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Eq. 10 from the start-field evaluation (delta_0 = 0.5, eta = 1): eta =
// sqrt(S^ang / S^str), 1 without angiography or when either sum is 0 or not
// finite; then the level's initial controller state.
__global__ void level_init_kernel(SolveState* S, const EvalResult* __restrict__ res, SolveCfg cfg) {
  double eta = 1.0;
  if (cfg.have_ang) {
    const double st = res->terms[0], an = res->terms[1];
    const double e = sqrt(an / st);
    if (st > 0.0 && an > 0.0 && isfinite(e)) eta = e;
  }
  S->n = cfg.n;
  S->m = cfg.m;
  S->max_iter = cfg.max_iter;
  S->max_ls = cfg.max_ls;
  S->max_evals = cfg.max_evals;
  S->gtol = cfg.gtol;
  S->ftol = cfg.ftol;
  S->mode = kModeInit;
  S->done = 0;
  S->status = 1;
  S->iters = S->evals = S->small = S->retried = S->ls = S->have_lo = 0;
  S->save_best = S->restore_best = S->branch = S->moved = 0;
  S->f = S->ft = S->fb = S->dg0 = S->a = S->lo = S->gmaxb = 0.0;
  S->hi = INFINITY;
  S->eta = eta;
  S->k = 0;
  S->spare = 0;
  S->ncand = 0;
  S->t_start = global_ns();
}

__global__ void level_stats_kernel(const SolveState* __restrict__ S, LevelStatsDev* out) {
  out->iters = S->iters;
  out->evals = S->evals;
  out->status = S->status;
  out->f = S->f;
  out->eta = S->eta;
  out->t_start = S->t_start;
  out->t_end = global_ns();
}

inline unsigned grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 4 * 152) b = 4 * 152;
  return (unsigned)b;
}

}  // namespace

// The products are float64 work, which this GPU runs at 1/64 of the float
// rate per SM: one block per SM, each with a contiguous share of the
// elements (fewer blocks on short vectors).
int solve_dots_blocks(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  const int sms = device_sm_count();
  if (b > sms) b = sms;
  if (b < 1) b = 1;
  return (int)b;
}

int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 152;
  if (dev < 64 && cached[dev] > 0) return cached[dev];
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  if (dev < 64) cached[dev] = sms;
  return sms;
}

cudaError_t launch_solve_trial(SolveState* S, const HistSet& H, const SolveVecs& V, EvalResult* res, double* partials,
                               unsigned* counter, cudaStream_t s) {
  trial_kernel<<<dim3(grid_for(V.plane), 6), kThreads, 0, s>>>(S, H, V, res, partials, counter);
  return cudaGetLastError();
}

cudaError_t launch_solve_dots(SolveState* S, const HistSet& H, int m, const SolveVecs& V, double* partials,
                              unsigned* counter, cudaStream_t s) {
  if (m < 1 || m > kMaxM) return cudaErrorInvalidValue;
  const int rows = (2 * (m + 1) + kChunk - 1) / kChunk;
  dots_kernel<<<dim3(solve_dots_blocks(V.n), rows), kThreads, 0, s>>>(S, H, V, partials, counter);
  return cudaGetLastError();
}

cudaError_t launch_solve_finish(const SolveState* S, const SolveVecs& V, cudaStream_t s) {
  finish_kernel<<<grid_for(V.n), kThreads, 0, s>>>(S, V);
  return cudaGetLastError();
}

cudaError_t launch_solve_level_init(SolveState* S, const EvalResult* res, SolveCfg cfg, cudaStream_t s) {
  level_init_kernel<<<1, 1, 0, s>>>(S, res, cfg);
  return cudaGetLastError();
}

cudaError_t launch_solve_level_stats(const SolveState* S, LevelStatsDev* out, cudaStream_t s) {
  level_stats_kernel<<<1, 1, 0, s>>>(S, out);
  return cudaGetLastError();
}



}  // namespace octmc
