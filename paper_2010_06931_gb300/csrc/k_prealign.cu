// Rough axial prealignment (Ploner et al., stage 1 of Sec. 2.1): the
// displacement field induced by per-B-scan axial offsets and tilts, and the
// reduction of the field's gradient to the parameters.
//
// Parameters of a level with w x h A-scans, [aX(h), tX(h), aY(w), tY(w)]:
// the X-fast B-scan j (a row) moves A-scan (i, j) axially by
// aX_j + tX_j (i - (w-1)/2), the Y-fast B-scan i (a column) moves (i, j) by
// aY_i + tY_i (j - (h-1)/2); transverse displacements are 0.  The tilt term
// fixes the three modes the data cannot see (a common x tilt, y tilt and
// x y twist of the frame, which both parameterisations can express), each
// weighted like the mean term M for the same displacement energy:
// T = 2 w vx sX^2 / h + 2 h vy sY^2 / w + 2 w h vx vy sT^2 / nT^2 with
// vx = (w^2-1)/12, vy = (h^2-1)/12, sX = sum tX, sY = sum tY,
// sT = sum_j tX_j (j - cy) + sum_i tY_i (i - cx), nT = h vy + w vx.
// All arithmetic is float64 with fixed reduction trees.
#include "common.cuh"

namespace octmc {
namespace {

constexpr int kThreads = 256;

__global__ void prm_to_disp_kernel(const double* __restrict__ prm, int w, int h, double* __restrict__ disp) {
  const int64_t plane = (int64_t)w * h, n = 6 * plane;
  const double cx = 0.5 * (w - 1), cy = 0.5 * (h - 1);
  const double *aX = prm, *tX = prm + h, *aY = prm + 2 * h, *tY = prm + 2 * h + w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int comp = (int)(e / plane);  // V * 3 + c
    const int64_t q = e - comp * plane;
    const int i = (int)(q % w), j = (int)(q / w);
    double v = 0.0;
    if (comp == 2) v = fma(tX[j], (double)i - cx, aX[j]);
    else if (comp == 5) v = fma(tY[i], (double)j - cy, aY[i]);
    disp[e] = v;
  }
}

// Fixed-order block sum of a double (result in every thread).
__device__ double block_sum_d(double v, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < kThreads / 32; i++) t += sm[i];
  return t;
}

// Block b < h: X B-scan (row) b; block h + b: Y B-scan (column) b.  Writes
// d f / d a and d f / d t of the B-scan (field gradient reduced along the
// fast axis, plus the tilt term's part); block 0 writes T to *T_out.
__global__ void __launch_bounds__(kThreads) grad_to_prm_kernel(const double* __restrict__ g, int w, int h,
                                                               const double* __restrict__ prm,
                                                               double* __restrict__ gprm, double* T_out) {
  __shared__ double sm[kThreads / 32];
  const int64_t plane = (int64_t)w * h;
  const bool isX = blockIdx.x < (unsigned)h;
  const int b = isX ? blockIdx.x : blockIdx.x - h;
  const int nf = isX ? w : h;
  const double c = 0.5 * (nf - 1);
  const double* gz = g + (isX ? 2 : 5) * plane;
  double ga = 0.0, gt = 0.0;
  for (int f = threadIdx.x; f < nf; f += kThreads) {
    const double v = isX ? gz[(int64_t)b * w + f] : gz[(int64_t)f * w + b];
    ga += v;
    gt = fma(v, (double)f - c, gt);
  }
  ga = block_sum_d(ga, sm);
  gt = block_sum_d(gt, sm);
  // the tilt functionals (same order in every block)
  const double cx = 0.5 * (w - 1), cy = 0.5 * (h - 1);
  double sX = 0.0, sY = 0.0, sT = 0.0, nT = 0.0;
  for (int k = threadIdx.x; k < h; k += kThreads) {
    const double t = prm[h + k], o = (double)k - cy;
    sX += t;
    sT = fma(t, o, sT);
    nT = fma(o, o, nT);
  }
  for (int k = threadIdx.x; k < w; k += kThreads) {
    const double t = prm[2 * h + w + k], o = (double)k - cx;
    sY += t;
    sT = fma(t, o, sT);
    nT = fma(o, o, nT);
  }
  sX = block_sum_d(sX, sm);
  sY = block_sum_d(sY, sm);
  sT = block_sum_d(sT, sm);
  nT = block_sum_d(nT, sm);
  const double vx = ((double)w * w - 1.0) / 12.0, vy = ((double)h * h - 1.0) / 12.0;
  const double lx = 2.0 * w * vx / h, ly = 2.0 * h * vy / w;
  const double lt = nT > 0.0 ? 2.0 * w * h * vx * vy / (nT * nT) : 0.0;
  if (threadIdx.x == 0) {
    if (isX) {
      gprm[b] = ga;
      gprm[h + b] = gt + 2.0 * lx * sX + 2.0 * lt * sT * ((double)b - cy);
    } else {
      gprm[2 * h + b] = ga;
      gprm[2 * h + w + b] = gt + 2.0 * ly * sY + 2.0 * lt * sT * ((double)b - cx);
    }
    if (blockIdx.x == 0) *T_out = lx * sX * sX + ly * sY * sY + lt * sT * sT;
  }
}

// One block: *out = a . b over n values (fixed order).
__global__ void __launch_bounds__(kThreads) prm_dot_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                           int n, double* out) {
  __shared__ double sm[kThreads / 32];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += kThreads) s = fma(a[k], b[k], s);
  s = block_sum_d(s, sm);
  if (threadIdx.x == 0) *out = s;
}

// Coarse (wc, hc) parameters to the fine level (wf, hf): fine B-scan b at
// (b - 1/2)/2 on the coarse level (clamped, linear); offsets double, tilts
// are kept.
__global__ void prm_prolong_kernel(const double* __restrict__ pc, int wc, int hc, double* __restrict__ pf, int wf,
                                   int hf) {
  const int n = 2 * (wf + hf);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int part, b;
    if (e < 2 * hf) {
      part = e / hf;
      b = e % hf;
    } else {
      part = 2 + (e - 2 * hf) / wf;
      b = (e - 2 * hf) % wf;
    }
    const int nc = part < 2 ? hc : wc;
    const double* c = pc + (part < 2 ? part * hc : 2 * hc + (part - 2) * wc);
    double x = fmin(fmax(0.5 * b - 0.25, 0.0), (double)(nc - 1));
    const int x0 = (int)x, x1 = min(x0 + 1, nc - 1);  // x >= 0: truncation is floor
    const double fx = x - x0;
    const double scale = (part % 2 == 0) ? 2.0 : 1.0;
    pf[e] = scale * ((1.0 - fx) * c[x0] + fx * c[x1]);
  }
}

inline unsigned grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 4 * 152) b = 4 * 152;
  return (unsigned)b;
}

}  // namespace

cudaError_t launch_prm_to_disp(const double* prm, int w, int h, double* disp, cudaStream_t s) {
  prm_to_disp_kernel<<<grid_for(6 * (int64_t)w * h), kThreads, 0, s>>>(prm, w, h, disp);
  return cudaGetLastError();
}

cudaError_t launch_grad_to_prm(const double* g, int w, int h, const double* prm, double* gprm, double* T_out,
                               cudaStream_t s) {
  grad_to_prm_kernel<<<(unsigned)(w + h), kThreads, 0, s>>>(g, w, h, prm, gprm, T_out);
  return cudaGetLastError();
}

cudaError_t launch_prm_dot(const double* a, const double* b, int n, double* out, cudaStream_t s) {
  prm_dot_kernel<<<1, kThreads, 0, s>>>(a, b, n, out);
  return cudaGetLastError();
}

cudaError_t launch_prm_prolong(const double* pc, int wc, int hc, double* pf, int wf, int hf, cudaStream_t s) {
  prm_prolong_kernel<<<grid_for(2 * (wf + hf)), kThreads, 0, s>>>(pc, wc, hc, pf, wf, hf);
  return cudaGetLastError();
}

}  // namespace octmc
