// One A-scan of an objective + gradient evaluation by one warp (Ploner et
// al., Eq. 1-10): the data term, then in the same warp the temporal
// regulariser along both scans' acquisition chains, the mean-term gradient
// and the float64 gradient, as used by the persistent small-level kernel.
#pragma once
#include "common.cuh"
#include "data.cuh"

namespace octmc {
namespace {

// Pseudo-Huber loss of a displacement difference and its derivative (the
// regulariser's L_epsR, as in the regulariser kernel).
__device__ __forceinline__ float huber_r(float x, float inv_eps, float* dl) {
  const float r = x * inv_eps;
  const float q = fmaf(r, r, 1.0f);
  const float is = rsqrtf(q);
  *dl = r * is;
  return __fdividef(x * r, fmaf(q, is, 1.0f));
}

// One A-scan of the evaluation by one warp: the data term (lanes 0..7 hold
// its outputs), then lanes 0..5 the regulariser terms, the mean-term
// gradient and the float64 gradient of component 3 V + c = lane; partial
// sums into acc (S^str, S^ang, R, grad . dir) and the running max |grad|.
template <typename T>
__device__ __forceinline__ void eval_ascan(const DataArgs& D, double* __restrict__ grad, const double* __restrict__ dir,
                                           int64_t p, int lane, float two_mu_s, float inv_eps_r, float alpha_d,
                                           double* acc, unsigned long long* gmx) {
  const LevelDev& L = D.L;
  const int64_t plane = (int64_t)L.w * L.h;
  const double* xt = D.disp;
  int base[6];
  float frac[6];
  split_displacement(xt, plane, p, (int)(p % L.w), (int)(p / L.w), L, lane, base, frac);
  const float out = data_value<T>(D, p, lane, base, frac);
  // lane 0: the A-scan's structural term, lane 1 its angiographic term,
  // lane 2 + q: the data-term gradient of component q
  const float gdat = __shfl_sync(0xffffffffu, out, (lane + 2) & 31);
  if (lane == 0) acc[0] += widen_exact(out);
  if (lane == 1) acc[1] += widen_exact(out);
  if (lane < 6) {
    const int V_ = lane / 3, c_ = lane % 3;
    const int nx = L.next[V_][p], pv = L.prev[V_][p];
    const double* dc = xt + (int64_t)(3 * V_ + c_) * plane;
    const double x = dc[p];
    float r = 0.f, gr = 0.f;
    if (nx >= 0) {  // pair (p, next) counted at its first sample
      float dl;
      const float wn = L.wnext[V_][p];
      r = wn * huber_r((float)(dc[nx] - x), inv_eps_r, &dl);  // float64 difference, rounded once
      gr = fmaf(-wn, dl, gr);
    }
    if (pv >= 0) {
      float dl;
      huber_r((float)(x - dc[pv]), inv_eps_r, &dl);
      gr = fmaf(L.wprev[V_][p], dl, gr);
    }
    const int64_t gi = (int64_t)(3 * V_ + c_) * plane + p;
    const double gw = widen_exact(gdat + fmaf(alpha_d, gr, two_mu_s));
    grad[gi] = gw;
    acc[2] += widen_exact(r);
    if (dir) acc[3] = fma(gw, dir[gi], acc[3]);  // line-search product in float64
    *gmx = max(*gmx, (unsigned long long)__double_as_longlong(gw) & 0x7fffffffffffffffull);
  }
}

}  // namespace
}  // namespace octmc
