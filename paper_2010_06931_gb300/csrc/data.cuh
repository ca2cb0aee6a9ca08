// Data term of one output A-scan by one warp (Ploner et al., Eq. 2-8),
// shared by the data-term kernels and the persistent small-level solve:
// the two displaced Catmull-Rom resamplings, the loss and its depth sums,
// the per-A-scan angiography, validity and delta, and the eight outputs.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "sample.cuh"

namespace octmc {
namespace {

// The data-term computation of output A-scan p by one warp (base and frac:
// the coordinate split of its 6 displacement values); the value of this
// lane's output (see data_core).
template <typename T>
__device__ __forceinline__ float data_value(const DataArgs& A, int64_t p, int lane, const int base[6],
                                            const float frac[6]) {
  const LevelDev& L = A.L;
  Vol VX, VY;
  setup_vol(VX, L.sx, L, base, frac);
  setup_vol(VY, L.sy, L, base + 3, frac + 3);

  const float inv_eps = 1.0f / A.eps_h;
  const bool ssd = (A.loss == OCTMC_LOSS_SSD);
  float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int nst = (L.d + kOutPerIter - 1) / kOutPerIter;
  for (int s = 0; s < nst; s++) {
    const int kb = s * kOutPerIter;
    float IX[4], IzX[4], IxX[4], IyX[4], IY[4], IzY[4], IxY[4], IyY[4];
    sample_block<T>(VX, kb, lane, L.dp, IX, IzX, IxX, IyX);
    sample_block<T>(VY, kb, lane, L.dp, IY, IzY, IxY, IyY);
    if (lane >= 1 && lane <= kOutLanes) {
#pragma unroll
      for (int o = 0; o < 4; o++) {
        const int k = kb + 4 * (lane - 1) + o;
        if (k < L.d) {
          const float R = IX[o] - IY[o];
          float Lv, dL;
          if (ssd) {
            Lv = R * R;
            dL = 2.0f * R;
          } else {
            // Eq. 4 as (R^2/eps) / (1 + sqrt(1 + (R/eps)^2)): no cancellation near 0
            const float rr = R * inv_eps;
            const float qv = fmaf(rr, rr, 1.0f);
            const float is = rsqrtf(qv);
            dL = rr * is;
            Lv = __fdividef(R * rr, fmaf(qv, is, 1.0f));
          }
          acc[0] += Lv;
          const float2 d2 = make_float2(dL, dL);
          float2 t = ffma2(d2, make_float2(IxX[o], IyX[o]), make_float2(acc[1], acc[2]));
          acc[1] = t.x; acc[2] = t.y;
          t = ffma2(d2, make_float2(IzX[o], IxY[o]), make_float2(acc[3], acc[4]));
          acc[3] = t.x; acc[4] = t.y;
          t = ffma2(d2, make_float2(IyY[o], IzY[o]), make_float2(acc[5], acc[6]));
          acc[5] = t.x; acc[6] = t.y;
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 7; c++) acc[c] = warp_sum(acc[c]);

  // ---- per-A-scan scalars (Eq. 6-8), float, every lane
  // Eq. 7: X validity along y at j + dy^X, Y validity along x at i + dx^Y,
  // by the zero-tangent Hermite interpolant (no overshoot: 0 <= delta <= delta_0)
  float vtx = 1.f, dvtx = 0.f, vty = 1.f, dvty = 0.f;
  if (L.vx) validity_hermite(L.vx, L.h, VX.by, frac[1], &vtx, &dvtx);
  if (L.vy) validity_hermite(L.vy, L.w, VY.bx, frac[3], &vty, &dvty);
  const float delta0 = (float)A.delta0;
  const float delta = delta0 * vtx * vty;  // Eq. 8
  const float d = (float)L.d;

  float La = 0.f, dLa = 0.f, aXx = 0.f, aXy = 0.f, aYx = 0.f, aYy = 0.f;
  if (L.ax) {
    // Eq. 6: the 16 taps of A^X (lanes 0..15) and of A^Y (lanes 16..31) at
    // the displaced transverse positions, then a butterfly within each half
    const bool isX = lane < 16;
    const float* img = isX ? L.ax : L.ay;
    const int a = lane & 3, b = (lane >> 2) & 3;
    float wa = 0.f, dwa = 0.f, wb = 0.f, dwb = 0.f;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const float wxq = isX ? VX.wx[q] : VY.wx[q], dwxq = isX ? VX.dwx[q] : VY.dwx[q];
      const float wyq = isX ? VX.wy[q] : VY.wy[q], dwyq = isX ? VX.dwy[q] : VY.dwy[q];
      if (a == q) { wa = wxq; dwa = dwxq; }
      if (b == q) { wb = wyq; dwb = dwyq; }
    }
    const int bxs = isX ? VX.bx : VY.bx, bys = isX ? VX.by : VY.by;
    const float sv = img[(int64_t)clampi(bys - 1 + b, L.h) * L.w + clampi(bxs - 1 + a, L.w)];
    float v = wa * wb * sv, vx = dwa * wb * sv, vy = wa * dwb * sv;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      v += __shfl_xor_sync(kFull, v, o);
      vx += __shfl_xor_sync(kFull, vx, o);
      vy += __shfl_xor_sync(kFull, vy, o);
    }
    const float ov = __shfl_xor_sync(kFull, v, 16);
    const float ovx = __shfl_xor_sync(kFull, vx, 16);
    const float ovy = __shfl_xor_sync(kFull, vy, 16);
    const float AX = (lane < 16) ? v : ov, AY = (lane < 16) ? ov : v;
    aXx = (lane < 16) ? vx : ovx; aXy = (lane < 16) ? vy : ovy;
    aYx = (lane < 16) ? ovx : vx; aYy = (lane < 16) ? ovy : vy;
    const float Ra = AX - AY;
    if (ssd) {
      La = Ra * Ra;
      dLa = 2.0f * Ra;
    } else {
      const float rr = Ra * inv_eps;
      const float qv = fmaf(rr, rr, 1.0f);
      const float is = rsqrtf(qv);
      dLa = rr * is;
      La = __fdividef(Ra * rr, fmaf(qv, is, 1.0f));
    }
  }

  // eight outputs of this A-scan, one per lane 0..7
  const float eta = (float)(A.eta_dev ? *A.eta_dev : A.eta);
  const float Lsum = acc[0];
  const float cs = eta * (1.0f - delta);
  const float ca = delta * d / eta * dLa;
  const float ddelta = -eta * Lsum + d * La / eta;
  float out;
  switch (lane) {
    case 0: out = (1.0f - delta) * Lsum; break;
    case 1: out = delta * d * La; break;
    case 2: out = cs * acc[1] + ca * aXx; break;
    case 3: out = cs * acc[2] + ca * aXy + ddelta * delta0 * dvtx * vty; break;
    case 4: out = cs * acc[3]; break;
    case 5: out = -cs * acc[4] - ca * aYx + ddelta * delta0 * vtx * dvty; break;
    case 6: out = -cs * acc[5] - ca * aYy; break;
    default: out = -cs * acc[6]; break;
  }
  return out;
}

// data_value written out: lane 0 the A-scan's structural term, lane 1 its
// angiographic term, lanes 2..7 the six gradient components (3 V + c).
template <typename T>
__device__ __forceinline__ void data_core(const DataArgs& A, int64_t p, int lane, const int base[6],
                                          const float frac[6]) {
  const float out = data_value<T>(A, p, lane, base, frac);
  const int64_t nasc = (int64_t)A.L.w * A.L.h;
  if (lane == 0) A.str_out[p] = out;
  else if (lane == 1) A.ang_out[p] = out;
  else if (lane < 8 && A.grad) A.grad[(int64_t)(lane - 2) * nasc + p] = out;
}

// Output A-scan p by one warp from the volumes in global memory.
template <typename T>
__device__ __forceinline__ void data_ascan(const DataArgs& A, int64_t p, int lane) {
  const LevelDev& L = A.L;
  const int64_t nasc = (int64_t)L.w * L.h;
  int base[6];
  float frac[6];
  split_displacement(A.disp, nasc, p, (int)(p % L.w), (int)(p / L.w), L, lane, base, frac);
  data_core<T>(A, p, lane, base, frac);
}

}  // namespace
}  // namespace octmc
