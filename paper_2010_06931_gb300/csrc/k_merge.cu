// Merging weights of the final resampling (Ploner et al., Sec. 2.1 last
// paragraphs, Sec. 2.5): per motion-corrected A-scan and scan, the sampling
// density (how many corrected A-scans sample the same input location), an
// exponentially decaying weight above the normal density, clipping and
// normalisation, and the validity-weighted en-face angiography merge.
//
// The density map is accumulated with 64-bit fixed-point integer atomics
// (weights in units of 2^-32), so its value does not depend on the order of
// the additions.
#include "common.cuh"
#include "sample.cuh"

namespace octmc {
namespace {

constexpr int kThreads = 256;
constexpr double kFix = 4294967296.0;  // 2^32

// Bilinear footprint of (u, v) = (i + dx, j + dy) clamped into the grid.
struct Foot {
  int x0, x1, y0, y1;
  float fx, fy;
};

__device__ __forceinline__ Foot footprint(const double* disp, int64_t n, int64_t p, int V, int i, int j, int w,
                                          int h) {
  Foot F;
  split_exact((unsigned long long)__double_as_longlong(disp[(int64_t)(3 * V + 0) * n + p]), i, 0, w - 1, &F.x0, &F.fx);
  split_exact((unsigned long long)__double_as_longlong(disp[(int64_t)(3 * V + 1) * n + p]), j, 0, h - 1, &F.y0, &F.fy);
  F.x1 = min(F.x0 + 1, w - 1);
  F.y1 = min(F.y0 + 1, h - 1);
  return F;
}

__global__ void splat_kernel(const double* __restrict__ disp, int w, int h, unsigned long long* counts) {
  const int64_t n = (int64_t)w * h;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int V = (int)(e / n);
    const int64_t p = e % n;
    const Foot F = footprint(disp, n, p, V, (int)(p % w), (int)(p / w), w, h);
    unsigned long long* c = counts + V * n;
    atomicAdd(c + (int64_t)F.y0 * w + F.x0, (unsigned long long)((1.0f - F.fx) * (1.0f - F.fy) * (float)kFix));
    atomicAdd(c + (int64_t)F.y0 * w + F.x1, (unsigned long long)(F.fx * (1.0f - F.fy) * (float)kFix));
    atomicAdd(c + (int64_t)F.y1 * w + F.x0, (unsigned long long)((1.0f - F.fx) * F.fy * (float)kFix));
    atomicAdd(c + (int64_t)F.y1 * w + F.x1, (unsigned long long)(F.fx * F.fy * (float)kFix));
  }
}

__device__ __forceinline__ float count_value(unsigned long long c) {
  // integer part + fraction (2^-32 units), without float64 arithmetic
  return (float)(unsigned)(c >> 32) + (float)(unsigned)(c & 0xffffffffull) * 2.3283064365386963e-10f;
}

__global__ void weights_kernel(LevelDev L, const double* __restrict__ disp, float beta, float tau,
                               const unsigned long long* __restrict__ counts, float* weights, float* angio) {
  const int w = L.w, h = L.h;
  const int64_t n = (int64_t)w * h;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % w), j = (int)(p / w);
    float wt[2];
    for (int V = 0; V < 2; V++) {
      const Foot F = footprint(disp, n, p, V, i, j, w, h);
      const unsigned long long* c = counts + V * n;
      const float rho = (1.0f - F.fx) * (1.0f - F.fy) * count_value(c[(int64_t)F.y0 * w + F.x0]) +
                        F.fx * (1.0f - F.fy) * count_value(c[(int64_t)F.y0 * w + F.x1]) +
                        (1.0f - F.fx) * F.fy * count_value(c[(int64_t)F.y1 * w + F.x0]) +
                        F.fx * F.fy * count_value(c[(int64_t)F.y1 * w + F.x1]);
      wt[V] = expf(-beta * fmaxf(0.0f, rho - 1.0f));
    }
    float c0 = wt[0] >= tau ? wt[0] : 0.0f, c1 = wt[1] >= tau ? wt[1] : 0.0f;
    if (c0 == 0.0f && c1 == 0.0f) {
      if (wt[0] >= wt[1]) c0 = 1.0f;
      else c1 = 1.0f;
    }
    const float wx = c0 / (c0 + c1), wy = c1 / (c0 + c1);
    if (weights) {
      weights[p] = wx;
      weights[n + p] = wy;
    }
    if (angio && L.ax) {
      // resampled en-face images (Eq. 6 positions) and validity (Eq. 7)
      float a[2], va[2] = {1.0f, 1.0f};
      for (int V = 0; V < 2; V++) {
        int bx, by;
        float tx, ty, wxv[4], dwx[4], wyv[4], dwy[4];
        split_exact((unsigned long long)__double_as_longlong(disp[(int64_t)(3 * V + 0) * n + p]), i, -4, w + 3, &bx, &tx);
        split_exact((unsigned long long)__double_as_longlong(disp[(int64_t)(3 * V + 1) * n + p]), j, -4, h + 3, &by, &ty);
        keys_weights(tx, wxv, dwx);
        keys_weights(ty, wyv, dwy);
        const float* img = V == 0 ? L.ax : L.ay;
        float s = 0.0f;
        for (int b = 0; b < 4; b++)
          for (int q = 0; q < 4; q++)
            s = fmaf(wxv[q] * wyv[b], img[(int64_t)clampi(by - 1 + b, h) * w + clampi(bx - 1 + q, w)], s);
        a[V] = s;
        const float* vv = V == 0 ? L.vx : L.vy;
        if (vv) {
          float dv;
          if (V == 0) validity_hermite(vv, h, by, ty, &va[V], &dv);
          else validity_hermite(vv, w, bx, tx, &va[V], &dv);
        }
      }
      const float a0 = fmaxf(0.0f, c0 * va[0]), a1 = fmaxf(0.0f, c1 * va[1]);
      angio[p] = (a0 + a1 > 0.0f) ? (a0 * a[0] + a1 * a[1]) / (a0 + a1) : 0.0f;
    }
  }
}

// Motion-corrected resampling and merging of one A-scan (warp): both scans
// resampled along depth at the displaced positions (the derivative parts of
// sample_block are dead code here), merged with the per-A-scan weights.
// Forward only, so it fits in 40 registers: 6 blocks (48 warps) per SM keep
// more loads in flight than the data kernel's 3.  vec4: d % 4 == 0 and every
// output 16-byte aligned, so a lane's 4 outputs go out as one 128-bit store.
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * kWarp, 6)
resample_merge_kernel(const LevelDev L, const double* __restrict__ disp, const float* __restrict__ weights,
                      float* merged, float* cx, float* cy, bool vec4) {
  const int64_t nasc = (int64_t)L.w * L.h;
  const int64_t p = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (p >= nasc) return;
  const int lane = threadIdx.x & 31;
  const int i = (int)(p % L.w), j = (int)(p / L.w);
  int base[6];
  float frac[6];
  split_displacement(disp, nasc, p, i, j, L, lane, base, frac);
  Vol VX, VY;
  setup_vol(VX, L.sx, L, base, frac);
  setup_vol(VY, L.sy, L, base + 3, frac + 3);
  const float wx = weights ? weights[p] : 0.5f, wy = weights ? weights[nasc + p] : 0.5f;
  for (int kb = 0; kb < L.d; kb += kOutPerIter) {
    float IX[4], IzX[4], IxX[4], IyX[4], IY[4], IzY[4], IxY[4], IyY[4];
    sample_block<T>(VX, kb, lane, L.dp, IX, IzX, IxX, IyX);
    sample_block<T>(VY, kb, lane, L.dp, IY, IzY, IxY, IyY);
    const int k0 = kb + 4 * (lane - 1);
    if (lane >= 1 && lane <= kOutLanes && k0 < L.d) {
      const int64_t e0 = p * L.d + k0;
      if (vec4) {  // k0 + 3 < d as d % 4 == 0
        if (merged)
          *reinterpret_cast<float4*>(merged + e0) =
              make_float4(fmaf(wx, IX[0], wy * IY[0]), fmaf(wx, IX[1], wy * IY[1]), fmaf(wx, IX[2], wy * IY[2]),
                          fmaf(wx, IX[3], wy * IY[3]));
        if (cx) *reinterpret_cast<float4*>(cx + e0) = make_float4(IX[0], IX[1], IX[2], IX[3]);
        if (cy) *reinterpret_cast<float4*>(cy + e0) = make_float4(IY[0], IY[1], IY[2], IY[3]);
      } else {
#pragma unroll
        for (int o = 0; o < 4; o++) {
          if (k0 + o < L.d) {
            if (merged) merged[e0 + o] = fmaf(wx, IX[o], wy * IY[o]);
            if (cx) cx[e0 + o] = IX[o];
            if (cy) cy[e0 + o] = IY[o];
          }
        }
      }
    }
  }
}

inline unsigned grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 65535) b = 65535;
  return (unsigned)b;
}

}  // namespace

cudaError_t launch_resample_merge(const LevelDev& L, const double* disp, const float* weights, float* merged,
                                  float* cx, float* cy, cudaStream_t s) {
  const int64_t nasc = (int64_t)L.w * L.h;
  const int64_t blocks = (nasc + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks <= 0) return cudaSuccess;
  auto a16 = [](const float* q) { return ((uintptr_t)q & 15u) == 0; };
  const bool vec4 = (L.d % 4 == 0) && a16(merged) && a16(cx) && a16(cy);
  const unsigned threads = kWarpsPerBlock * kWarp;
  if (L.dtype == OCTMC_BF16)
    resample_merge_kernel<__nv_bfloat16><<<(unsigned)blocks, threads, 0, s>>>(L, disp, weights, merged, cx, cy, vec4);
  else if (L.dtype == OCTMC_F16)
    resample_merge_kernel<__half><<<(unsigned)blocks, threads, 0, s>>>(L, disp, weights, merged, cx, cy, vec4);
  else
    resample_merge_kernel<float><<<(unsigned)blocks, threads, 0, s>>>(L, disp, weights, merged, cx, cy, vec4);
  return cudaGetLastError();
}

cudaError_t launch_merge_weights(const LevelDev& L, const double* disp, double beta, double tau,
                                 unsigned long long* counts, float* weights, float* angio, cudaStream_t s) {
  const int64_t n = (int64_t)L.w * L.h;
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * 2 * n, s);
  if (e != cudaSuccess) return e;
  splat_kernel<<<grid_for(2 * n), kThreads, 0, s>>>(disp, L.w, L.h, counts);
  weights_kernel<<<grid_for(n), kThreads, 0, s>>>(L, disp, (float)beta, (float)tau, counts, weights, angio);
  return cudaGetLastError();
}

}  // namespace octmc
