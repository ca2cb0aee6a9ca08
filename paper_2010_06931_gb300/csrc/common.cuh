// Internal declarations shared by the CUDA translation units of liboctmc.
// Device helpers, kernel argument structs and launcher prototypes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "octmc.h"

namespace octmc {

constexpr int kWarp = 32;

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

// Keys cubic-convolution kernel with a = -1/2 (the Catmull-Rom spline, i.e.
// cubic Hermite interpolation with central-difference tangents): weights of
// the samples at n-1, n, n+1, n+2 for a point n + t, expanded in powers of t
// and evaluated by Horner's rule, plus their t-derivatives.
__device__ __forceinline__ void keys_weights(float t, float w[4], float dw[4]) {
  w[0] = t * fmaf(t, fmaf(-0.5f, t, 1.0f), -0.5f);
  w[1] = fmaf(t * t, fmaf(1.5f, t, -2.5f), 1.0f);
  w[2] = t * fmaf(t, fmaf(-1.5f, t, 2.0f), 0.5f);
  w[3] = (t * t) * fmaf(0.5f, t, -0.5f);
  dw[0] = fmaf(t, fmaf(-1.5f, t, 2.0f), -0.5f);
  dw[1] = t * fmaf(4.5f, t, -5.0f);
  dw[2] = fmaf(t, fmaf(-4.5f, t, 4.0f), 0.5f);
  dw[3] = t * fmaf(1.5f, t, -1.0f);
}

// Validity line v (n samples) at b + t, 0 <= t < 1 (Ploner et al., Sec. 2.2,
// Eq. 7): the cubic Hermite interpolant with zero tangents at the nodes,
// v_b + (v_{b+1} - v_b) (3 t^2 - 2 t^3), edge samples replicated.  It is C^1
// and never leaves the range of its two nodes, so delta (Eq. 8) stays within
// [0, delta_0] next to invalid B-scans.
__device__ __forceinline__ void validity_hermite(const float* v, int n, int b, float t, float* val,
                                                 float* dval) {
  const float p0 = v[clampi(b, n)], p1 = v[clampi(b + 1, n)];
  const float dp = p1 - p0;
  *val = fmaf(dp, (t * t) * fmaf(-2.0f, t, 3.0f), p0);
  *dval = dp * (6.0f * t) * (1.0f - t);
}

// Exact split of u = off + v, v a double given by its bit pattern and off an
// integer, into floor(u) and the fraction u - floor(u) as a float (mantissa
// truncated to 24 bits), after clamping u into the integer range [lo, hi].
// Integer instructions only: double arithmetic runs at 1/64 of the float
// rate on this GPU and has a long latency.  NaN maps to lo, -inf to lo, +inf
// to hi, |v| >= 2^31 to the nearer bound; float-subnormal fractions to 0.
__device__ __forceinline__ void split_exact(unsigned long long bits, int off, int lo, int hi, int* base,
                                            float* t) {
  const unsigned h32 = (unsigned)(bits >> 32);
  const bool neg = (h32 >> 31) != 0;
  const int ex = (int)((h32 >> 20) & 0x7ffu);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (ex == 0x7ff) {  // inf or NaN
    *base = (m == 0ull && !neg) ? hi : lo;
    *t = 0.f;
    return;
  }
  if (ex >= 1023 + 31) {
    *base = neg ? lo : hi;
    *t = 0.f;
    return;
  }
  int sh;  // |v| = m * 2^-sh, sh >= 22
  if (ex == 0) {
    sh = 1074;
  } else {
    m |= 1ull << 52;
    sh = 1075 - ex;
  }
  unsigned long long ip, fb;
  if (sh >= 64) {
    ip = 0ull;
    fb = m;
  } else {
    ip = m >> sh;
    fb = m & ((1ull << sh) - 1ull);
  }
  float f = 0.f;  // fb * 2^-sh, built from its bits
  if (fb != 0ull) {
    const int lz = __clzll((long long)fb);
    const int pos = 63 - lz;  // leading bit of fb
    const unsigned mant = (unsigned)((fb << lz) >> 40);  // top 24 bits, leading 1 included
    const int ef = pos - sh + 127;
    if (ef > 0) f = __uint_as_float(((unsigned)ef << 23) | (mant & 0x7fffffu));
  }
  int b;
  float tt;
  const int ipi = (int)ip;
  if (!neg) {
    b = off + ipi;
    tt = f;
  } else if (f > 0.f) {
    b = off - ipi - 1;
    tt = 1.0f - f;
  } else {
    b = off - ipi;
    tt = 0.f;
  }
  if (b < lo) {
    b = lo;
    tt = 0.f;
  } else if (b > hi || (b == hi && tt > 0.f)) {
    b = hi;
    tt = 0.f;
  }
  *base = b;
  *t = tt;
}

// Float to double by assembling the bits (exact for normal floats and zero;
// float subnormals become signed zero; inf and NaN stay inf and NaN).
__device__ __forceinline__ double widen_exact(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned m = u & 0x7fffffu;
  unsigned hi, lo;
  if (e == 0u) {
    hi = sign;
    lo = 0u;
  } else if (e == 255u) {
    hi = sign | 0x7ff00000u | (m >> 3);
    lo = m << 29;
  } else {
    hi = sign | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// Double to float by truncating the mantissa (integer instructions only):
// values below the float normal range become signed zero, values beyond it
// infinity; NaN stays NaN.
__device__ __forceinline__ float narrow_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h = (unsigned)(b >> 32);
  const unsigned sign = h & 0x80000000u;
  const int e = (int)((h >> 20) & 0x7ffu);
  const unsigned mant = (unsigned)((b >> 29) & 0x7fffffu);
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (mant | ((b & 0xFFFFFFFFFFFFFull) ? 1u : 0u)));
  const int ef = e - 1023 + 127;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)ef << 23) | mant);
}

// Deterministic warp sum (xor butterfly; every lane ends with the total).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- level data
// One pyramid level on the device.  Volumes are [h][w][dp] with dp = d
// rounded up to a multiple of 4; the pad samples [d, dp) repeat sample d-1,
// so aligned 4-sample groups inside [0, dp) read clamp-to-edge values.
struct LevelDev {
  int w, h, d, dp;
  int dtype;  // octmc_dtype of sx, sy (float32, bfloat16 or float16 samples)
  void* sx;
  void* sy;
  float* ax;  // [h][w] or null
  float* ay;
  float* vx;  // [h] or null
  float* vy;  // [w] or null
  // time-ordered chain of each volume (the temporal regulariser's pairs):
  // for A-scan p, the previous/next A-scan in acquisition order (-1: none)
  // and the weight of the pair (prev, p) / (p, next).
  int* prev[2];
  int* next[2];
  float* wprev[2];
  float* wnext[2];
};

// Arguments of the data-term kernel (Eq. 2-8 per A-scan).
struct DataArgs {
  LevelDev L;
  const double* disp;  // [2][3][h][w]
  float* str_out;      // [h*w]: (1 - delta) sum_k L(R_ijk)
  float* ang_out;      // [h*w]: delta d L(R_ij(A))
  float* grad;         // [2][3][h][w] data-term gradient, or null
  double eta;          // Eq. 9
  const double* eta_dev;  // if not null: eta is read here (set on the device, Eq. 10)
  double delta0;       // Eq. 8 (0 without angiography)
  float eps_h;         // Eq. 4
  int loss;            // octmc_loss
};

// Output of the final reduction of one evaluation.
struct EvalResult {
  double terms[6];  // S^str, S^ang, R, M, f, eta
  double gdir;      // grad . dir (line search), 0 if no dir
  double msum[3];   // sum over both volumes of each displacement component
};

// ---------------------------------------------------------------- device-resident level solve
// L-BFGS with the weak-Wolfe bisection line search of one pyramid level
// (Sec. 2.1), driven on the device: one CUDA graph per level whose WHILE
// node evaluates one trial point per iteration; the regulariser kernel's
// last block takes the line-search decision, and an IF node runs the
// accepted-step branch (history pair, products, compact-form direction).
constexpr int kMaxM = 32;
constexpr int kModeInit = 0;    // evaluate the start point of the level
constexpr int kModeTrial = 1;   // evaluate x + a dir
constexpr int kModeAccept = 2;  // branch: take the accepted trial, new pair, new direction
constexpr int kModeRetry = 3;   // branch: history dropped, direction -g
struct __align__(16) SolveState {  // 16-byte aligned: copied to shared memory with 16-byte vectors
  // configuration (set by the host before each launch)
  int64_t n;
  int m, max_iter, max_ls, max_evals;
  double gtol, ftol;
  // line-search controller
  int mode, done, status, iters, evals, small, retried, ls, have_lo, save_best, restore_best, branch;
  int moved;                    // the last decision took a new iterate (init or accepted step)
  double f, ft, fb, dg0, a, lo, hi;
  double gmaxb;                 // max |g| at the line search's best Armijo point
  double eta;                   // Eq. 10 at the level's start field
  unsigned long long t_start;   // %globaltimer at the level's start (ns)
  // history: buffer ids 0..m; order[0..k) oldest first; cand the vectors of the last products
  int k, spare, ncand;
  int order[kMaxM + 1];
  int cand[kMaxM + 1];
  double SY[(kMaxM + 1) * (kMaxM + 1)];
  double YY[(kMaxM + 1) * (kMaxM + 1)];
  double sg[kMaxM + 1], yg[kMaxM + 1];
  double gg, gmax;
  // direction: dir = cg g + sum_j coef[j] h_j, h_j = S[hid[j] / 2] (even) or Y[hid[j] / 2] (odd)
  double cg;
  int nc;
  int hid[2 * kMaxM + 2];
  double coef[2 * kMaxM + 2];
  double dots[2 * (2 * kMaxM + 2) + 3];
};

// Configuration of a level solve, set on the device at the level's start.
struct SolveCfg {
  int64_t n;
  int m, max_iter, max_ls, max_evals;
  double gtol, ftol;
  int have_ang;
};

// Per-level statistics written on the device at the level's end.
struct LevelStatsDev {
  int iters, evals, status, pad;
  double f, eta;
  unsigned long long t_start, t_end;
};

// The history buffers of one level solve.
struct HistSet {
  double* S[kMaxM + 1];
  double* Y[kMaxM + 1];
};

struct RegArgs {
  LevelDev L;
  const double* disp;
  double* grad;           // may be null: output gradient (data + R + M)
  const float* gdata;     // data-term gradient from the data kernel (if grad)
  const double* dir;      // may be null: then gdir = 0
  const float* str_in;    // [h*w]
  const float* ang_in;    // [h*w]
  double alpha, eps_r, mu, eta;
  const double* eta_dev;  // if not null: eta is read here
  EvalResult* result;     // device
  double* partials;       // [grid][8] scratch
  unsigned* counter;      // zero-initialised, reset by the last block
  SolveState* ctl;        // may be null: the line-search decision of a device-resident solve
  cudaGraphConditionalHandle h_branch;  // set with ctl: runs the accepted-step branch
  cudaGraphConditionalHandle h_while;   // set with ctl: continues the level's loop
};

// Batched evaluation of several problems ("slots") in one launch per
// kernel.  Data kernel: slot s owns the A-scans [begin[s], begin[s+1]) of
// the launch.  Reduction kernels: slot s owns the blocks [b0[s], b0[s+1]) --
// the same number and partition of blocks as a launch for that slot alone,
// so its sums do not depend on the other slots.  The arguments travel in the
// kernel parameter block (at most 32 KB).
constexpr int kMaxSlots = 48;
struct DataMulti {
  int nslots;
  int64_t total;
  int64_t begin[kMaxSlots + 1];
  DataArgs da[kMaxSlots];
};
struct MsumSlot {
  const double* disp;
  int64_t plane;
  EvalResult* res;
  double* partials;
  unsigned* counter;
};
struct MsumMulti {
  int nslots;
  int b0[kMaxSlots + 1];
  MsumSlot sl[kMaxSlots];
};
struct RegMulti {
  int nslots;
  int b0[kMaxSlots + 1];
  RegArgs ra[kMaxSlots];
};

// ---------------------------------------------------------------- launchers
// all slots of one data launch share the storage dtype
cudaError_t launch_data_multi(const DataMulti& M, int dtype, cudaStream_t s);
cudaError_t launch_msum_multi(const MsumMulti& M, cudaStream_t s);
cudaError_t launch_reg_multi(const RegMulti& M, cudaStream_t s);
cudaError_t launch_data(const DataArgs& a, cudaStream_t s);
cudaError_t launch_msum(const double* disp, int64_t plane, EvalResult* res, double* partials,
                        unsigned* counter, cudaStream_t s);
cudaError_t launch_reg(const RegArgs& a, cudaStream_t s);
int reg_grid_blocks(int64_t n_ascans);
int msum_grid_blocks();

// Rough axial prealignment (stage 1 of Sec. 2.1).
cudaError_t launch_prm_to_disp(const double* prm, int w, int h, double* disp, cudaStream_t s);
cudaError_t launch_grad_to_prm(const double* g, int w, int h, const double* prm, double* gprm, double* T_out,
                               cudaStream_t s);
cudaError_t launch_prm_dot(const double* a, const double* b, int n, double* out, cudaStream_t s);
cudaError_t launch_prm_prolong(const double* pc, int wc, int hc, double* pf, int wf, int hf, cudaStream_t s);

// Final resampling / merging (Sec. 2.1, 2.5).
cudaError_t launch_resample_merge(const LevelDev& L, const double* disp, const float* weights, float* merged,
                                  float* cx, float* cy, cudaStream_t s);
cudaError_t launch_merge_weights(const LevelDev& L, const double* disp, double beta, double tau,
                                 unsigned long long* counts, float* weights, float* angio, cudaStream_t s);

cudaError_t launch_pad_depth(float* vol, int64_t columns, int d, int dp, cudaStream_t s);
cudaError_t launch_pyr_volume(const float* in, int w, int h, int d, int dp, float* out, int w2,
                              int h2, int d2, int dp2, cudaStream_t s);
cudaError_t launch_pyr_image(const float* in, int w, int h, float* out, cudaStream_t s);
cudaError_t launch_pyr_line(const float* in, int n, float* out, cudaStream_t s);
cudaError_t launch_prolong(const double* coarse, int wc, int hc, double* fine, int wf, int hf,
                           cudaStream_t s);
cudaError_t launch_unpad_depth(const void* vol, int dtype, int64_t columns, int d, int dp, float* out,
                               cudaStream_t s);
cudaError_t launch_convert(const float* in, void* out, int dtype, int64_t n, cudaStream_t s);

// L-BFGS vector kernels.  The iterate x, the gradient g, the direction and
// the history pairs (s, y) are float64, and so are all products and sums.
constexpr int kMaxHist = 66;  // 2 (m + 1) history vectors for m <= 32
// Dot products of K history vectors with up to two probes q0 (the newest y)
// and q1 (a gradient); a null probe reads as 0.
// Outputs: [2k] = h_k . q0, [2k+1] = h_k . q1 (k < K), [2K] = q0 . q0,
// [2K+1] = q1 . q1, [2K+2] = max |q1| (exact).
struct HistDots {
  const double* h[kMaxHist];
  int K;
  const double* q0;
  const double* q1;
};
__host__ __device__ inline int hist_dots_outputs(int K) { return 2 * K + 3; }
// out = cg g + sum_k c_k h_k.
struct HistComb {
  const double* g;
  double cg;
  const double* h[kMaxHist];
  double c[kMaxHist];
  int K;
};
int hist_dots_blocks(int64_t n);
cudaError_t launch_hist_dots(const HistDots& hd, int64_t n, double* partials, unsigned* counter, double* out,
                             cudaStream_t s);
cudaError_t launch_hist_comb(const HistComb& hc, int64_t n, double* out, cudaStream_t s);
// s = x1 - x0, y = g1 - g0.
cudaError_t launch_sub2(const double* x1, const double* x0, const double* g1, const double* g0,
                        double* s_out, double* y_out, int64_t n, cudaStream_t st);
cudaError_t launch_axpy(const double* x, double a, const double* d, double* out, int64_t n,
                        cudaStream_t s);

// Device-resident level solve (k_solve.cu; the line-search decision itself
// runs in the regulariser kernel, solve.cuh).
// The vectors of one level solve (device, n = 6 w h float64 each; plane = w h).
struct SolveVecs {
  double *x, *g;    // iterate and its gradient
  double *xt, *gt;  // trial point and its gradient
  double *xb, *gb;  // the line search's best Armijo point
  double* dir;      // search direction
  int64_t n, plane;
};
cudaError_t launch_solve_trial(SolveState* S, const HistSet& H, const SolveVecs& V, EvalResult* res, double* partials,
                               unsigned* counter, cudaStream_t s);
cudaError_t launch_solve_dots(SolveState* S, const HistSet& H, int m, const SolveVecs& V, double* partials,
                              unsigned* counter, cudaStream_t s);
cudaError_t launch_solve_finish(const SolveState* S, const SolveVecs& V, cudaStream_t s);

// The persistent small-level solve: one cooperative kernel runs the whole
// loop of a level (k_level.cu).  S holds the level's initial state (from
// level_init_kernel) on entry and its final state on exit; x the start field
// on entry and the result on exit.
struct LevelArgs {
  SolveState* S;
  HistSet H;
  SolveVecs V;
  DataArgs D;             // the data term at V.xt (eta read through D.eta_dev)
  double alpha, eps_r, mu;
  double* part;           // scratch: level_part_doubles(grid) doubles
  unsigned* bar;          // [2] grid-barrier arrivals and generation, zero on entry
  int* err;               // 0 on entry; set when a grid barrier times out
};
int level_grid(int dtype);              // blocks of the cooperative launch (0: not available)
int64_t level_part_doubles(int grid);   // scratch size
cudaError_t launch_level_persistent(const LevelArgs& A, int dtype, cudaStream_t s);
cudaError_t launch_barrier_probe(unsigned* bar, int* err, int extra, cudaStream_t s);
int solve_dots_blocks(int64_t n);
int device_sm_count();  // SMs of the current device (queried once per device)
cudaError_t launch_solve_level_init(SolveState* S, const EvalResult* res, SolveCfg cfg, cudaStream_t s);
cudaError_t launch_solve_level_stats(const SolveState* S, LevelStatsDev* out, cudaStream_t s);

}  // namespace octmc
