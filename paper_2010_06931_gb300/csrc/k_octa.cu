// Angiography preprocessing of one scan (Ploner et al., Sec. 2.2 and 2.3):
// saccade validity of the B-scans and the en-face OCTA projection.
//
//   bscan_sum_kernel     per-B-scan sums (every sample widened exactly and
//                        added in float64, fixed tree per block): mean
//                        decorrelation of each B-scan, and the OCT sums for
//                        the OCT threshold
//   validity_kernel      mu, sigma of the B-scan means, the 3-sigma test and
//                        the +-2 B-scan dilation (one block, float64)
//   median3_kernel       3x3x3 median per voxel (edge replicated): the 9
//                        depth triples sorted, 14 samples provably on either
//                        side of the median dropped, forgetful selection of
//                        the median of the 13 others
//   rank15_kernel        3rd smallest of 15 samples along x or y (edge
//                        replicated) with a 3-deep insertion network
//   radix_hist_kernel /  exact order statistics of the filtered voxels of the
//   radix_pick_kernel    valid B-scans by 3 passes of 11-bit (last 10-bit)
//                        radix selection on order-preserving integer keys
//                        (integer histograms: deterministic)
//   finish_kernel        percentiles (linear interpolation), the mask cut
//                        and the OCT threshold (float64, one thread)
//   project_kernel       per A-scan (one warp): mean of the OCTA voxels whose
//                        filtered value is below the cut and whose OCT value
//                        is above the threshold
//   bscan_median_kernel  median of each B-scan's en-face values (bitonic sort
//                        in shared memory) subtracted from them
//   replace_kernel       invalid B-scans take the nearest valid one
//
// Volumes are float32 [h][w][d], depth contiguous.  B-scans of an X-fast
// scan (fast_axis 0) are the rows j, of a Y-fast scan the columns i.
#include <algorithm>
#include <cmath>
#include <new>

#include "common.cuh"

namespace octmc {
namespace {

constexpr int kT = 256;
constexpr int kRadixBins = 2048;
constexpr int kTargets = 4;  // order statistics: floor/ceil positions of two percentiles

struct Select {
  // per target: rank (0-based) among the selected voxels, key prefix found so
  // far, and the value once known
  long long rank[kTargets];
  unsigned prefix[kTargets];
  float value[kTargets];
  double pos[2];      // q (n - 1) of the two percentiles
  double p[2];        // the percentiles
  double cut;         // p_lo + thresh (p_hi - p_lo)
  double t_oct;       // OCT threshold
  float cut_f;        // smallest float >= cut: x < cut  <=>  x < cut_f
  float toct_f;       // largest float <= t_oct: x > t_oct <=> x > toct_f
};

__device__ __forceinline__ int64_t ascan_of(int w, int fast_axis, int b, int f) {
  return fast_axis == 0 ? (int64_t)b * w + f : (int64_t)f * w + b;
}

// ---------------------------------------------------------------- sums
// Block b sums the voxels of B-scan b (nf columns of d samples).
constexpr int kSumThreads = 1024;
__global__ void __launch_bounds__(kSumThreads) bscan_sum_kernel(const float* __restrict__ vol, int w, int h, int d,
                                                                int fast_axis, double* __restrict__ sums) {
  const int b = blockIdx.x;
  const int nf = fast_axis == 0 ? w : h;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // every sample widened and added in float64 (no float rounding); two
  // independent chains per lane for the float64 latency
  double acc0 = 0.0, acc1 = 0.0;
  for (int f = warp; f < nf; f += kSumThreads / 32) {
    const float* col = vol + ascan_of(w, fast_axis, b, f) * d;
    int k = lane;
    for (; k + 32 < d; k += 64) {
      acc0 += widen_exact(col[k]);
      acc1 += widen_exact(col[k + 32]);
    }
    if (k < d) acc0 += widen_exact(col[k]);
  }
  double acc = warp_sum(acc0 + acc1);
  __shared__ double sm[kSumThreads / 32];
  if (lane == 0) sm[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kSumThreads / 32; i++) t += sm[i];
    sums[b] = t;
  }
}

// One block: means, mu, sigma, saturation test, validity.
__global__ void __launch_bounds__(1024) validity_kernel(const double* __restrict__ sums, int nb, double per,
                                                        float* __restrict__ v, double* __restrict__ means) {
  __shared__ double sm[32];
  __shared__ double s_mu, s_sig;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a += sums[b] / per;
  a = warp_sum(a);
  if (lane == 0) sm[warp] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nw; i++) t += sm[i];
    s_mu = t / nb;
  }
  __syncthreads();
  const double mu = s_mu;
  double q = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double m = sums[b] / per;
    q += (m - mu) * (m - mu);
  }
  q = warp_sum(q);
  __syncthreads();
  if (lane == 0) sm[warp] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nw; i++) t += sm[i];
    s_sig = sqrt(t / nb);
  }
  __syncthreads();
  const double lim = mu + 3.0 * s_sig;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    bool ok = true;
    for (int o = -2; o <= 2; o++) {
      const int c = b + o;
      if (c >= 0 && c < nb && sums[c] / per > lim) ok = false;
    }
    v[b] = ok ? 1.0f : 0.0f;
    if (means) means[b] = sums[b] / per;
  }
}

// ---------------------------------------------------------------- filters
__device__ __forceinline__ int clampn(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

__device__ __forceinline__ void cmpx(float& a, float& b) {  // a <- min, b <- max
  const float mn = fminf(a, b), mx = fmaxf(a, b);
  a = mn;
  b = mx;
}

// Forgetful selection of the median of N = W + M values: a[0..W-1] holds
// the first W, rest[0..M-1] the others (W = (N+1)/2 + 1).  Each step moves
// the minimum of the current window a[LO..W-1] to a[LO] and its maximum to
// a[W-1], forgets both (the window start advances, the next value replaces
// the maximum); three candidates remain and the median is their middle one.
template <int W, int M, int LO = 0>
__device__ __forceinline__ void forget_steps(float (&a)[W], const float (&rest)[M]) {
  if constexpr (LO < M) {
    cmpx(a[LO], a[W - 1]);
#pragma unroll
    for (int i = LO + 1; i < W - 1; i++) {
      cmpx(a[LO], a[i]);
      cmpx(a[i], a[W - 1]);
    }
    a[W - 1] = rest[LO];
    forget_steps<W, M, LO + 1>(a, rest);
  }
}

__device__ __forceinline__ float median3_of(float x, float y, float z) {
  return fmaxf(fminf(x, y), fminf(fmaxf(x, y), z));
}

// The median of the 27 samples v[9][3] (9 neighbour columns, 3 depths):
// sort each column's 3 samples into (low, mid, high); in the order of the
// 27 values the 5 smallest lows and the 2 smallest mids lie at or below the
// median (each has at least 14 values at or above it), the 5 largest highs
// and the 2 largest mids at or above it, so the median is that of the 13
// others -- the 4 largest lows, the middle 5 mids, the 4 smallest highs --
// found by forgetful selection.  150 compare-exchanges instead of 192 for
// forgetful selection over all 27.
__device__ __forceinline__ float median27(float (&v)[9][3]) {
  float lo[9], mid[9], hi[9];
#pragma unroll
  for (int c = 0; c < 9; c++) {
    cmpx(v[c][0], v[c][1]);
    cmpx(v[c][1], v[c][2]);
    cmpx(v[c][0], v[c][1]);
    lo[c] = v[c][0];
    mid[c] = v[c][1];
    hi[c] = v[c][2];
  }
  // the 4 largest lows to lo[5..8]
#pragma unroll
  for (int e = 8; e >= 5; e--)
#pragma unroll
    for (int i = 0; i < e; i++) cmpx(lo[i], lo[e]);
  // the 4 smallest highs to hi[0..3]
#pragma unroll
  for (int b = 0; b <= 3; b++)
#pragma unroll
    for (int i = b + 1; i < 9; i++) cmpx(hi[b], hi[i]);
  // the 2 smallest mids to mid[0..1], the 2 largest to mid[7..8]
#pragma unroll
  for (int r = 0; r < 2; r++) {
    cmpx(mid[r], mid[8 - r]);
#pragma unroll
    for (int i = r + 1; i < 8 - r; i++) {
      cmpx(mid[r], mid[i]);
      cmpx(mid[i], mid[8 - r]);
    }
  }
  float a[8] = {lo[5], lo[6], lo[7], lo[8], mid[2], mid[3], mid[4], mid[5]};
  const float rest[5] = {mid[6], hi[0], hi[1], hi[2], hi[3]};
  forget_steps<8, 5>(a, rest);
  return median3_of(a[5], a[6], a[7]);
}

// Stencil launch geometry: block (32 depths, 8 columns i), grid (depth
// chunks, column chunks, rows j): no index division, warps read 128 coalesced
// bytes along depth, and blocks run in volume order so the rows a wave reads
// stay in L2.
constexpr int kSx = 32, kSy = 8;

__global__ void __launch_bounds__(kSx * kSy) median3_kernel(const float* __restrict__ in, int w, int h, int d,
                                                            float* __restrict__ out) {
  const int k = blockIdx.x * kSx + threadIdx.x;
  const int i = blockIdx.y * kSy + threadIdx.y;
  const int j = blockIdx.z;
  if (k >= d || i >= w) return;
  // offsets of the clamped neighbours from the voxel, per axis
  const int64_t row = (int64_t)w * d;
  const float* c0 = in + (int64_t)j * row + (int64_t)i * d + k;
  const int64_t ro[3] = {(int64_t)(clampn(j - 1, h) - j) * row, 0, (int64_t)(clampn(j + 1, h) - j) * row};
  const int co[3] = {(clampn(i - 1, w) - i) * d, 0, (clampn(i + 1, w) - i) * d};
  const int ko[3] = {k > 0 ? -1 : 0, 0, k + 1 < d ? 1 : 0};
  float v[9][3];
#pragma unroll
  for (int dj = 0; dj < 3; dj++)
#pragma unroll
    for (int di = 0; di < 3; di++) {
      const float* col = c0 + ro[dj] + co[di];
#pragma unroll
      for (int dk = 0; dk < 3; dk++) v[dj * 3 + di][dk] = __ldg(col + ko[dk]);
    }
  out[((int64_t)j * w + i) * d + k] = median27(v);
}

template <int AXIS>
__global__ void __launch_bounds__(kSx * kSy) rank15_kernel(const float* __restrict__ in, int w, int h, int d,
                                                           float* __restrict__ out) {
  const int k = blockIdx.x * kSx + threadIdx.x;
  const int i = blockIdx.y * kSy + threadIdx.y;
  const int j = blockIdx.z;
  if (k >= d || i >= w) return;
  const int64_t row = (int64_t)w * d;
  const float* c0 = in + (int64_t)j * row + (int64_t)i * d + k;
  float a1 = INFINITY, a2 = INFINITY, a3 = INFINITY;
#pragma unroll
  for (int o = -7; o <= 7; o++) {
    const int64_t off = AXIS == 0 ? (int64_t)((clampn(i + o, w) - i) * d) : (int64_t)(clampn(j + o, h) - j) * row;
    const float x = __ldg(c0 + off);
    const float t = fmaxf(a1, x);
    a1 = fminf(a1, x);
    const float u = fmaxf(a2, t);
    a2 = fminf(a2, t);
    a3 = fminf(a3, u);
  }
  out[((int64_t)j * w + i) * d + k] = a3;
}

// ---------------------------------------------------------------- selection
__device__ __forceinline__ unsigned order_key(float x) {
  const unsigned u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_value(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// digit pass `pass` (0: bits 31..21, 1: 20..10, 2: 9..0)
__device__ __forceinline__ int digit_shift(int pass) { return pass == 0 ? 21 : (pass == 1 ? 10 : 0); }
__device__ __forceinline__ unsigned digit_mask(int pass) { return pass == 2 ? 0x3ffu : 0x7ffu; }

// Histogram of the current digit of the selected voxels whose higher digits
// equal each target's prefix.  hist [kTargets][kRadixBins].  Targets with
// the same prefix share one count (slot[t] = first target with t's
// prefix).  Each thread takes runs of kRun consecutive voxels and counts
// equal consecutive digits in registers before one shared atomic per run of
// equal digits: the filtered volume is smooth along depth, so the few hot
// bins of the leading digit (sign and exponent) are not hammered.
constexpr int kRun = 16;
__global__ void __launch_bounds__(kT) radix_hist_kernel(const float* __restrict__ vol, int w, int h, int d,
                                                        int fast_axis, const float* __restrict__ v, int any_valid,
                                                        const Select* __restrict__ sel, int pass,
                                                        unsigned* __restrict__ hist) {
  __shared__ unsigned sh[kTargets][kRadixBins];
  for (int t = threadIdx.x; t < kTargets * kRadixBins; t += kT) (&sh[0][0])[t] = 0u;
  __syncthreads();
  const int sft = digit_shift(pass);
  const unsigned msk = digit_mask(pass);
  unsigned pre[kTargets];
  int slot[kTargets];
#pragma unroll
  for (int t = 0; t < kTargets; t++) {
    pre[t] = sel->prefix[t];
    slot[t] = t;
    for (int u = t - 1; u >= 0; u--)
      if (pre[u] == pre[t]) slot[t] = u;
  }
  const int hs = sft + (pass == 2 ? 10 : 11);  // the bits above the digit start at hs
  const int64_t n = (int64_t)w * h * d;
  const int64_t nrun = (n + kRun - 1) / kRun;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrun; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = r * kRun;
    int64_t p = e / d;
    int k = (int)(e - p * d);
    unsigned cur[kTargets], cnt[kTargets];
#pragma unroll
    for (int t = 0; t < kTargets; t++) {
      cur[t] = 0u;
      cnt[t] = 0u;
    }
    // whether the current A-scan's B-scan is selected (recomputed when the
    // run crosses into the next A-scan)
    auto selected = [&](int64_t pp) {
      const int b = fast_axis == 0 ? (int)(pp / w) : (int)(pp % w);
      return !(any_valid && v[b] == 0.0f);
    };
    bool sel_p = selected(p);
    // the run's samples first (independent loads, 128-bit when the run is
    // whole and aligned), then the counting
    float x[kRun];
    if (e + kRun <= n && ((reinterpret_cast<uintptr_t>(vol + e) & 15u) == 0)) {
#pragma unroll
      for (int c = 0; c < kRun / 4; c++) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(vol + e) + c);
        x[4 * c] = f.x;
        x[4 * c + 1] = f.y;
        x[4 * c + 2] = f.z;
        x[4 * c + 3] = f.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < kRun; q++) x[q] = e + q < n ? __ldg(vol + e + q) : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < kRun; q++, e++) {
      if (e >= n) break;
      if (sel_p) {
        const unsigned key = order_key(x[q]);
        const unsigned dig = (key >> sft) & msk;
        const unsigned hi = hs >= 32 ? 0u : (key >> hs);
#pragma unroll
        for (int t = 0; t < kTargets; t++) {
          if (slot[t] != t || hi != pre[t]) continue;
          if (cnt[t] && dig != cur[t]) {
            atomicAdd(&sh[t][cur[t]], cnt[t]);
            cnt[t] = 0u;
          }
          cur[t] = dig;
          cnt[t]++;
        }
      }
      if (++k == d) {
        k = 0;
        p++;
        if (q + 1 < kRun && e + 1 < n) sel_p = selected(p);
      }
    }
#pragma unroll
    for (int t = 0; t < kTargets; t++)
      if (cnt[t]) atomicAdd(&sh[t][cur[t]], cnt[t]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kTargets * kRadixBins; i += kT) {
    const int t = i / kRadixBins, bin = i % kRadixBins;
    const int st = t == 0 ? slot[0] : (t == 1 ? slot[1] : (t == 2 ? slot[2] : slot[3]));
    const unsigned c = sh[st][bin];
    if (c) atomicAdd(hist + i, c);
  }
}

// One block of kRadixBins / 2 threads: for each target, the bin holding its
// rank (block-wide exclusive scan of the histogram, each thread owning two
// consecutive bins); prefix and rank are narrowed to that bin.  After the
// last pass the key is complete.  Clears the histograms for the next pass.
constexpr int kPickThreads = kRadixBins / 2;
__global__ void __launch_bounds__(kPickThreads) radix_pick_kernel(Select* sel, unsigned* hist, int pass) {
  __shared__ unsigned long long warp_tot[kPickThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned nbins = digit_mask(pass) + 1u;
  const int width = pass == 2 ? 10 : 11;
  for (int t = 0; t < kTargets; t++) {
    unsigned* hb = hist + t * kRadixBins;
    const unsigned c0 = 2 * tid < (int)nbins ? hb[2 * tid] : 0u;
    const unsigned c1 = 2 * tid + 1 < (int)nbins ? hb[2 * tid + 1] : 0u;
    // inclusive scan of the pair sums within the warp, then across warps
    unsigned long long x = (unsigned long long)c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    unsigned long long before = 0;
    for (int i = 0; i < warp; i++) before += warp_tot[i];
    const unsigned long long incl = before + x;
    const unsigned long long excl = incl - c0 - c1;
    const long long r = sel->rank[t];
    __syncthreads();  // every thread has read rank[t] and warp_tot before they change
    if ((long long)excl <= r && r < (long long)incl) {
      const bool first = r < (long long)(excl + c0);
      const unsigned bin = 2 * tid + (first ? 0u : 1u);
      sel->prefix[t] = (sel->prefix[t] << width) | bin;
      sel->rank[t] = r - (long long)(first ? excl : excl + c0);
      if (pass == 2) sel->value[t] = key_value(sel->prefix[t]);
    }
    __syncthreads();
  }
  for (int i = tid; i < kTargets * kRadixBins; i += kPickThreads) hist[i] = 0u;
}

__global__ void finish_kernel(Select* sel, const double* __restrict__ oct_sums, const float* __restrict__ v,
                              int nb, int any_valid, double per_bscan, double thresh, double t_oct_in) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = 0; q < 2; q++) {
    const double pos = sel->pos[q];
    const double lo = floor(pos);
    const double a = sel->value[2 * q], b = sel->value[2 * q + 1];
    sel->p[q] = a + (pos - lo) * (b - a);
  }
  sel->cut = sel->p[0] + thresh * (sel->p[1] - sel->p[0]);
  double t = t_oct_in;
  if (isnan(t)) {
    double s = 0.0, cnt = 0.0;
    for (int b = 0; b < nb; b++)
      if (!any_valid || v[b] != 0.0f) {
        s += oct_sums[b];
        cnt += per_bscan;
      }
    t = s / cnt;
  }
  sel->t_oct = t;
  // float bounds that reproduce the double comparisons exactly
  float c = (float)sel->cut;  // round to nearest
  if ((double)c < sel->cut) c = nextafterf(c, INFINITY);
  else if ((double)nextafterf(c, -INFINITY) >= sel->cut) c = nextafterf(c, -INFINITY);
  sel->cut_f = c;
  float o = (float)t;
  if ((double)o > t) o = nextafterf(o, -INFINITY);
  sel->toct_f = o;
}

// ---------------------------------------------------------------- projection
// One warp per A-scan.
__global__ void __launch_bounds__(kT) project_kernel(const float* __restrict__ A, const float* __restrict__ S,
                                                     const float* __restrict__ F, int64_t nasc, int d,
                                                     const Select* __restrict__ sel, float* __restrict__ E,
                                                     unsigned long long* __restrict__ kept) {
  const int lane = threadIdx.x & 31;
  const float cut = sel->cut_f, to = sel->toct_f;
  for (int64_t p = (int64_t)blockIdx.x * (kT / 32) + (threadIdx.x >> 5); p < nasc;
       p += (int64_t)gridDim.x * (kT / 32)) {  // warp-uniform
    float s = 0.f;
    int c = 0;
    for (int k = lane; k < d; k += 32) {
      const int64_t e = p * d + k;
      if (F[e] < cut && S[e] > to) {
        s += A[e];
        c++;
      }
    }
    s = warp_sum(s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
      E[p] = c ? s / (float)c : 0.0f;
      if (c) atomicAdd(kept, (unsigned long long)c);
    }
  }
}

// One block per B-scan: bitonic sort of its en-face values in shared memory,
// median, subtraction.  nf <= kMaxFast.
constexpr int kMaxFast = 4096;
__global__ void __launch_bounds__(1024) bscan_median_kernel(float* __restrict__ E, int w, int h, int fast_axis) {
  __shared__ float s[kMaxFast];
  const int b = blockIdx.x;
  const int nf = fast_axis == 0 ? w : h;
  int np = 1;
  while (np < nf) np <<= 1;
  for (int f = threadIdx.x; f < np; f += blockDim.x) s[f] = f < nf ? E[ascan_of(w, fast_axis, b, f)] : INFINITY;
  __syncthreads();
  for (int size = 2; size <= np; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int jx = i ^ stride;
        if (jx > i) {
          const bool up = (i & size) == 0;
          const float x = s[i], y = s[jx];
          if ((x > y) == up) {
            s[i] = y;
            s[jx] = x;
          }
        }
      }
      __syncthreads();
    }
  const double med = (nf & 1) ? (double)s[nf / 2] : 0.5 * ((double)s[nf / 2 - 1] + (double)s[nf / 2]);
  __syncthreads();
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    float* e = E + ascan_of(w, fast_axis, b, f);
    *e = (float)((double)*e - med);
  }
}

// Block per B-scan: an invalid B-scan copies the nearest valid one (lower
// index on a tie) from src (the subtracted image before replacement).
__global__ void replace_kernel(const float* __restrict__ src, float* __restrict__ E, int w, int h, int fast_axis,
                               const float* __restrict__ v) {
  const int b = blockIdx.x;
  const int nb = fast_axis == 0 ? h : w, nf = fast_axis == 0 ? w : h;
  if (v[b] != 0.0f) return;
  int best = -1;
  for (int dist = 1; dist < nb && best < 0; dist++) {
    if (b - dist >= 0 && v[b - dist] != 0.0f) best = b - dist;
    else if (b + dist < nb && v[b + dist] != 0.0f) best = b + dist;
  }
  if (best < 0) return;
  for (int f = threadIdx.x; f < nf; f += blockDim.x) E[ascan_of(w, fast_axis, b, f)] = src[ascan_of(w, fast_axis, best, f)];
}

// One element (or A-scan) per thread (warp) up to the grid limit.
inline unsigned grid_for(int64_t n, int per = kT) {
  int64_t b = (n + per - 1) / per;
  if (b < 1) b = 1;
  if (b > 0x7fffffff) b = 0x7fffffff;
  return (unsigned)b;
}

struct CudaErr {
  cudaError_t e;
};
inline void ck(cudaError_t e) {
  if (e != cudaSuccess) throw CudaErr{e};
}

}  // namespace
}  // namespace octmc

using namespace octmc;

extern "C" int octmc_saccade_validity(const float* octa, int w, int h, int d, int fast_axis, float* v,
                                      double* means, void* stream) {
  if (!octa || !v || w < 1 || h < 1 || d < 1 || (fast_axis != 0 && fast_axis != 1)) return OCTMC_ERR_INVALID_ARG;
  const cudaStream_t st = (cudaStream_t)stream;
  const int nb = fast_axis == 0 ? h : w, nf = fast_axis == 0 ? w : h;
  double* sums = nullptr;
  try {
    ck(cudaMallocAsync(&sums, sizeof(double) * nb, st));
    bscan_sum_kernel<<<nb, kSumThreads, 0, st>>>(octa, w, h, d, fast_axis, sums);
    ck(cudaGetLastError());
    validity_kernel<<<1, 1024, 0, st>>>(sums, nb, (double)nf * d, v, means);
    ck(cudaGetLastError());
    ck(cudaFreeAsync(sums, st));
    ck(cudaStreamSynchronize(st));
  } catch (const CudaErr&) {
    cudaGetLastError();
    return OCTMC_ERR_CUDA;
  }
  return OCTMC_OK;
}

extern "C" int octmc_enface(const float* octa, const float* oct, int w, int h, int d, int fast_axis, const float* v,
                            double q_lo, double q_hi, double thresh, double t_oct, float* enface, float* filtered,
                            double* info, void* stream) {
  if (!octa || !oct || !v || !enface || w < 1 || h < 1 || d < 1 || (fast_axis != 0 && fast_axis != 1))
    return OCTMC_ERR_INVALID_ARG;
  if (!(q_lo >= 0.0 && q_lo <= 1.0 && q_hi >= 0.0 && q_hi <= 1.0) || !std::isfinite(thresh))
    return OCTMC_ERR_INVALID_ARG;
  const int nb = fast_axis == 0 ? h : w, nf = fast_axis == 0 ? w : h;
  if (nf > kMaxFast || h > 65535 || (w + 7) / 8 > 65535) return OCTMC_ERR_UNSUPPORTED;
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t nvox = (int64_t)w * h * d, nasc = (int64_t)w * h;
  // validity is needed on the host for the selected-voxel count
  float* vh = nullptr;
  float *m3 = nullptr, *r1 = nullptr, *r2 = nullptr, *esrc = nullptr;
  double* osum = nullptr;
  Select* sel = nullptr;
  unsigned* hist = nullptr;
  unsigned long long* kept = nullptr;
  int rc = OCTMC_OK;
  try {
    vh = new float[nb];
    ck(cudaMemcpyAsync(vh, v, sizeof(float) * nb, cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    int nvalid = 0;
    for (int b = 0; b < nb; b++) nvalid += vh[b] != 0.0f;
    const int any = nvalid > 0;
    const long long nsel = (long long)(any ? nvalid : nb) * nf * d;
    Select s0{};
    const double qs[2] = {q_lo, q_hi};
    for (int q = 0; q < 2; q++) {
      s0.pos[q] = qs[q] * (double)(nsel - 1);
      const long long lo = (long long)std::floor(s0.pos[q]);
      s0.rank[2 * q] = lo;
      s0.rank[2 * q + 1] = lo + 1 < nsel ? lo + 1 : lo;
    }
    ck(cudaMallocAsync(&m3, sizeof(float) * nvox, st));
    ck(cudaMallocAsync(&r1, sizeof(float) * nvox, st));
    r2 = filtered;
    if (!r2) ck(cudaMallocAsync(&r2, sizeof(float) * nvox, st));
    ck(cudaMallocAsync(&osum, sizeof(double) * nb, st));
    ck(cudaMallocAsync(&sel, sizeof(Select), st));
    ck(cudaMallocAsync(&hist, sizeof(unsigned) * kTargets * kRadixBins, st));
    ck(cudaMallocAsync(&kept, sizeof(unsigned long long), st));
    ck(cudaMallocAsync(&esrc, sizeof(float) * nasc, st));
    ck(cudaMemcpyAsync(sel, &s0, sizeof(Select), cudaMemcpyHostToDevice, st));
    ck(cudaMemsetAsync(hist, 0, sizeof(unsigned) * kTargets * kRadixBins, st));
    ck(cudaMemsetAsync(kept, 0, sizeof(unsigned long long), st));
    // filters
    const dim3 sb(kSx, kSy), sg((unsigned)((d + kSx - 1) / kSx), (unsigned)((w + kSy - 1) / kSy), (unsigned)h);
    median3_kernel<<<sg, sb, 0, st>>>(octa, w, h, d, m3);
    ck(cudaGetLastError());
    // fast axis first, then the slow axis
    if (fast_axis == 0) rank15_kernel<0><<<sg, sb, 0, st>>>(m3, w, h, d, r1);
    else rank15_kernel<1><<<sg, sb, 0, st>>>(m3, w, h, d, r1);
    ck(cudaGetLastError());
    if (fast_axis == 0) rank15_kernel<1><<<sg, sb, 0, st>>>(r1, w, h, d, r2);
    else rank15_kernel<0><<<sg, sb, 0, st>>>(r1, w, h, d, r2);
    ck(cudaGetLastError());
    // percentiles of the filtered voxels of the valid B-scans
    for (int pass = 0; pass < 3; pass++) {
      // streaming, no reuse: a resident-size grid, each block one shared histogram
      const unsigned hb = (unsigned)std::min<int64_t>((nvox / kRun + kT) / kT, 152 * 8);
      radix_hist_kernel<<<hb, kT, 0, st>>>(r2, w, h, d, fast_axis, v, any, sel, pass, hist);
      ck(cudaGetLastError());
      radix_pick_kernel<<<1, kPickThreads, 0, st>>>(sel, hist, pass);
      ck(cudaGetLastError());
    }
    // OCT threshold from the per-B-scan OCT sums, cut, projection
    if (std::isnan(t_oct)) {
      bscan_sum_kernel<<<nb, kSumThreads, 0, st>>>(oct, w, h, d, fast_axis, osum);
      ck(cudaGetLastError());
    }
    finish_kernel<<<1, 32, 0, st>>>(sel, osum, v, nb, any, (double)nf * d, thresh, t_oct);
    ck(cudaGetLastError());
    project_kernel<<<grid_for(nasc, kT / 32), kT, 0, st>>>(octa, oct, r2, nasc, d, sel, enface, kept);
    ck(cudaGetLastError());
    bscan_median_kernel<<<nb, 1024, 0, st>>>(enface, w, h, fast_axis);
    ck(cudaGetLastError());
    if (any && nvalid < nb) {
      ck(cudaMemcpyAsync(esrc, enface, sizeof(float) * nasc, cudaMemcpyDeviceToDevice, st));
      replace_kernel<<<nb, 256, 0, st>>>(esrc, enface, w, h, fast_axis, v);
      ck(cudaGetLastError());
    }
    if (info) {
      Select s1;
      unsigned long long kh = 0;
      ck(cudaMemcpyAsync(&s1, sel, sizeof(Select), cudaMemcpyDeviceToHost, st));
      ck(cudaMemcpyAsync(&kh, kept, sizeof(kh), cudaMemcpyDeviceToHost, st));
      ck(cudaStreamSynchronize(st));
      info[0] = s1.p[0];
      info[1] = s1.p[1];
      info[2] = s1.t_oct;
      info[3] = (double)kh;
    }
  } catch (const CudaErr&) {
    cudaGetLastError();
    rc = OCTMC_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    rc = OCTMC_ERR_OOM;
  }
  if (m3) cudaFreeAsync(m3, st);
  if (r1) cudaFreeAsync(r1, st);
  if (r2 && r2 != filtered) cudaFreeAsync(r2, st);
  if (osum) cudaFreeAsync(osum, st);
  if (sel) cudaFreeAsync(sel, st);
  if (hist) cudaFreeAsync(hist, st);
  if (kept) cudaFreeAsync(kept, st);
  if (esrc) cudaFreeAsync(esrc, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == OCTMC_OK) rc = OCTMC_ERR_CUDA;
  delete[] vh;
  return rc;
}
