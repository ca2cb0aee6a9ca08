// Data term of the registration objective (Ploner et al., Eq. 2-8) and its
// gradient with respect to every A-scan displacement, fused in one kernel.
//
// For output A-scan (i, j) and each scan V in {X, Y}, the volume S^V is
// sampled along depth at (i + dx^V, j + dy^V, k + dz^V), k = 0..d-1, with
// the separable 4x4x4 Catmull-Rom interpolator (clamp-to-edge).  The
// residual R_k = I^X(k) - I^Y(k) (Eq. 2) goes through the loss (Eq. 4, or
// squared differences) and is summed over k (Eq. 3/5); the derivative of
// the sum with respect to the 6 displacement values of the A-scan is reduced
// over depth in the same pass.  The en-face angiography term (Eq. 6), the
// resampled validity (Eq. 7) and delta (Eq. 8) are per-A-scan scalars.
//
// Mapping: one warp per output A-scan.  Depth is processed in blocks of 116
// outputs; lane L (1..29) owns outputs kb + 4(L-1) .. +3.  Each lane loads
// one aligned group of 4 input samples from each of the 16 transverse
// neighbour columns with one 128-bit load per column (coalesced along depth
// across the warp), forms the transverse interpolant T and its x/y
// derivatives Tx, Ty for those 4 input depths, and gets the 3 neighbouring
// input depths the 4-tap axial filter needs from the adjacent lanes by
// shuffles.  Lanes 0, 30 and 31 only supply those halo values.  Per-A-scan
// sums are reduced with a fixed butterfly, so results are deterministic.
#include "common.cuh"

namespace octmc {
namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kOutLanes = 29;
constexpr int kOutPerIter = 4 * kOutLanes;
constexpr unsigned kFull = 0xffffffffu;

struct Vol {
  const float4* base;  // the volume as 4-sample groups
  unsigned roff[4];    // row offsets (in groups) of the 4 neighbour rows
  unsigned coff[4];    // column offsets (in groups) of the 4 neighbour columns
  float wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
  int q, r;            // floor(dz) = 4 q + r, 0 <= r < 4
  int bx, by;          // floor of the transverse coordinates
};

__device__ __forceinline__ void setup_vol(Vol& V, const float* vol, const LevelDev& L, int i, int j,
                                          double dx, double dy, double dz) {
  float tx, ty, tz;
  split_coord((double)i + dx, L.w, &V.bx, &tx);
  split_coord((double)j + dy, L.h, &V.by, &ty);
  // Along depth every output k shares floor(dz) and the fraction; beyond
  // |dz| > d + 4 all taps are edge samples, so dz is clamped to +-(d + 8).
  double dzc = fmin(fmax(dz, -(double)L.d - 8.0), (double)L.d + 8.0);
  double fz = floor(dzc);
  int kz0 = (int)fz;
  tz = (float)(dzc - fz);
  V.q = kz0 >> 2;  // arithmetic shift: floor division by 4
  V.r = kz0 & 3;
  keys_weights(tx, V.wx, V.dwx);
  keys_weights(ty, V.wy, V.dwy);
  keys_weights(tz, V.wz, V.dwz);
  const unsigned nq = (unsigned)(L.dp >> 2);
#pragma unroll
  for (int a = 0; a < 4; a++) {
    V.roff[a] = (unsigned)clampi(V.by - 1 + a, L.h) * (unsigned)L.w * nq;
    V.coff[a] = (unsigned)clampi(V.bx - 1 + a, L.w) * nq;
  }
  V.base = reinterpret_cast<const float4*>(vol);
}

__device__ __forceinline__ void fma4(float4& acc, float w, const float4& s) {
  acc.x = fmaf(w, s.x, acc.x);
  acc.y = fmaf(w, s.y, acc.y);
  acc.z = fmaf(w, s.z, acc.z);
  acc.w = fmaf(w, s.w, acc.w);
}

__device__ __forceinline__ float4 bcast(float v) { return make_float4(v, v, v, v); }

// Axial 4-tap filter for the lane's 4 outputs.  e[1..4] hold the lane's
// own input group, e[0] the last sample of lane-1's group, e[5..8] lane+1's
// group and e[9] the first sample of lane+2's.  Output o, tap c reads
// e[R + o + c], where R = floor(dz) mod 4.
template <int R>
__device__ __forceinline__ void axial(const float4& T, const float4& Tx, const float4& Ty,
                                      const float wz[4], const float dwz[4], float I[4], float Iz[4],
                                      float Ix[4], float Iy[4]) {
  float e[10], ex[10], ey[10];
  e[1] = T.x; e[2] = T.y; e[3] = T.z; e[4] = T.w;
  ex[1] = Tx.x; ex[2] = Tx.y; ex[3] = Tx.z; ex[4] = Tx.w;
  ey[1] = Ty.x; ey[2] = Ty.y; ey[3] = Ty.z; ey[4] = Ty.w;
  if (R == 0) {
    e[0] = __shfl_up_sync(kFull, T.w, 1);
    ex[0] = __shfl_up_sync(kFull, Tx.w, 1);
    ey[0] = __shfl_up_sync(kFull, Ty.w, 1);
  }
  e[5] = __shfl_down_sync(kFull, T.x, 1);
  ex[5] = __shfl_down_sync(kFull, Tx.x, 1);
  ey[5] = __shfl_down_sync(kFull, Ty.x, 1);
  e[6] = __shfl_down_sync(kFull, T.y, 1);
  ex[6] = __shfl_down_sync(kFull, Tx.y, 1);
  ey[6] = __shfl_down_sync(kFull, Ty.y, 1);
  if (R >= 1) {
    e[7] = __shfl_down_sync(kFull, T.z, 1);
    ex[7] = __shfl_down_sync(kFull, Tx.z, 1);
    ey[7] = __shfl_down_sync(kFull, Ty.z, 1);
  }
  if (R >= 2) {
    e[8] = __shfl_down_sync(kFull, T.w, 1);
    ex[8] = __shfl_down_sync(kFull, Tx.w, 1);
    ey[8] = __shfl_down_sync(kFull, Ty.w, 1);
  }
  if (R == 3) {
    e[9] = __shfl_down_sync(kFull, T.x, 2);
    ex[9] = __shfl_down_sync(kFull, Tx.x, 2);
    ey[9] = __shfl_down_sync(kFull, Ty.x, 2);
  }
#pragma unroll
  for (int o = 0; o < 4; o++) {
    float a = 0.f, az = 0.f, ax = 0.f, ay = 0.f;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      a = fmaf(wz[c], e[R + o + c], a);
      az = fmaf(dwz[c], e[R + o + c], az);
      ax = fmaf(wz[c], ex[R + o + c], ax);
      ay = fmaf(wz[c], ey[R + o + c], ay);
    }
    I[o] = a; Iz[o] = az; Ix[o] = ax; Iy[o] = ay;
  }
}

// Interpolated values (and their displacement derivatives) of one volume
// at the lane's 4 outputs of the depth block starting at kb.
__device__ __forceinline__ void sample_block(const Vol& V, int kb, int lane, int dp, float I[4],
                                             float Iz[4], float Ix[4], float Iy[4]) {
  const int qk = kb + 4 * V.q + 4 * (lane - 1);  // first input depth of the lane's group
  const unsigned qc = (unsigned)(min(max(qk, 0), dp - 4) >> 2);
  float4 T = bcast(0.f), Tx = bcast(0.f), Ty = bcast(0.f);
#pragma unroll
  for (int b = 0; b < 4; b++) {
    float4 U = bcast(0.f), Ux = bcast(0.f);
#pragma unroll
    for (int a = 0; a < 4; a++) {
      const float4 s = __ldg(V.base + (V.roff[b] + V.coff[a] + qc));
      fma4(U, V.wx[a], s);
      fma4(Ux, V.dwx[a], s);
    }
    fma4(T, V.wy[b], U);
    fma4(Tx, V.wy[b], Ux);
    fma4(Ty, V.dwy[b], U);
  }
  // groups entirely before sample 0 / after the last sample hold the edge value
  if (qk < 0) {
    T = bcast(T.x); Tx = bcast(Tx.x); Ty = bcast(Ty.x);
  } else if (qk >= dp) {
    T = bcast(T.w); Tx = bcast(Tx.w); Ty = bcast(Ty.w);
  }
  switch (V.r) {
    case 0: axial<0>(T, Tx, Ty, V.wz, V.dwz, I, Iz, Ix, Iy); break;
    case 1: axial<1>(T, Tx, Ty, V.wz, V.dwz, I, Iz, Ix, Iy); break;
    case 2: axial<2>(T, Tx, Ty, V.wz, V.dwz, I, Iz, Ix, Iy); break;
    default: axial<3>(T, Tx, Ty, V.wz, V.dwz, I, Iz, Ix, Iy); break;
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * kWarp)
data_kernel(const DataArgs A) {
  const LevelDev& L = A.L;
  const int lane = threadIdx.x & 31;
  const int64_t nasc = (int64_t)L.w * L.h;
  const int64_t p = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (p >= nasc) return;  // warp-uniform
  const int i = (int)(p % L.w), j = (int)(p / L.w);

  double dX[3], dY[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    dX[c] = A.disp[(0 * 3 + c) * nasc + p];
    dY[c] = A.disp[(1 * 3 + c) * nasc + p];
  }
  Vol VX, VY;
  setup_vol(VX, L.sx, L, i, j, dX[0], dX[1], dX[2]);
  setup_vol(VY, L.sy, L, i, j, dY[0], dY[1], dY[2]);

  const float inv_eps = 1.0f / A.eps_h;
  const bool ssd = (A.loss == OCTMC_LOSS_SSD);
  float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int kb = 0; kb < L.d; kb += kOutPerIter) {
    float IX[4], IzX[4], IxX[4], IyX[4], IY[4], IzY[4], IxY[4], IyY[4];
    sample_block(VX, kb, lane, L.dp, IX, IzX, IxX, IyX);
    sample_block(VY, kb, lane, L.dp, IY, IzY, IxY, IyY);
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
          acc[1] = fmaf(dL, IxX[o], acc[1]);
          acc[2] = fmaf(dL, IyX[o], acc[2]);
          acc[3] = fmaf(dL, IzX[o], acc[3]);
          acc[4] = fmaf(dL, IxY[o], acc[4]);
          acc[5] = fmaf(dL, IyY[o], acc[5]);
          acc[6] = fmaf(dL, IzY[o], acc[6]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 7; c++) acc[c] = warp_sum(acc[c]);
  if (lane != 0) return;

  // ---- per-A-scan scalars (Eq. 6-8), lane 0
  const double d = (double)L.d;
  double vtx = 1.0, dvtx = 0.0, vty = 1.0, dvty = 0.0;
  if (L.vx) {  // Eq. 7: X validity along y at j + dy^X (same weights as S^X in y)
    float v = 0.f, dv = 0.f;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const float s = L.vx[clampi(VX.by - 1 + b, L.h)];
      v = fmaf(VX.wy[b], s, v);
      dv = fmaf(VX.dwy[b], s, dv);
    }
    vtx = v; dvtx = dv;
  }
  if (L.vy) {  // Y validity along x at i + dx^Y
    float v = 0.f, dv = 0.f;
#pragma unroll
    for (int a = 0; a < 4; a++) {
      const float s = L.vy[clampi(VY.bx - 1 + a, L.w)];
      v = fmaf(VY.wx[a], s, v);
      dv = fmaf(VY.dwx[a], s, dv);
    }
    vty = v; dvty = dv;
  }
  const double delta0 = A.delta0;
  const double delta = delta0 * vtx * vty;  // Eq. 8

  double La = 0.0, dLa = 0.0, gAX[2] = {0.0, 0.0}, gAY[2] = {0.0, 0.0};
  if (L.ax) {  // Eq. 6: en-face residual at the displaced transverse positions
    float aX = 0.f, aXx = 0.f, aXy = 0.f, aY = 0.f, aYx = 0.f, aYy = 0.f;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int rX = clampi(VX.by - 1 + b, L.h), rY = clampi(VY.by - 1 + b, L.h);
#pragma unroll
      for (int a = 0; a < 4; a++) {
        const float sX = L.ax[(int64_t)rX * L.w + clampi(VX.bx - 1 + a, L.w)];
        const float sY = L.ay[(int64_t)rY * L.w + clampi(VY.bx - 1 + a, L.w)];
        aX = fmaf(VX.wx[a] * VX.wy[b], sX, aX);
        aXx = fmaf(VX.dwx[a] * VX.wy[b], sX, aXx);
        aXy = fmaf(VX.wx[a] * VX.dwy[b], sX, aXy);
        aY = fmaf(VY.wx[a] * VY.wy[b], sY, aY);
        aYx = fmaf(VY.dwx[a] * VY.wy[b], sY, aYx);
        aYy = fmaf(VY.wx[a] * VY.dwy[b], sY, aYy);
      }
    }
    const double Ra = (double)aX - (double)aY;
    if (ssd) {
      La = Ra * Ra;
      dLa = 2.0 * Ra;
    } else {
      const double rr = Ra / (double)A.eps_h;
      const double s = sqrt(1.0 + rr * rr);
      dLa = rr / s;
      La = (Ra * rr) / (1.0 + s);
    }
    gAX[0] = aXx; gAX[1] = aXy; gAY[0] = aYx; gAY[1] = aYy;
  }

  const double Lsum = acc[0];
  A.str_out[p] = (1.0 - delta) * Lsum;
  A.ang_out[p] = delta * d * La;
  if (A.grad) {
    const double eta = A.eta;
    const double cs = eta * (1.0 - delta);
    const double ca = delta * d / eta * dLa;
    const double ddelta = -eta * Lsum + d * La / eta;
    double* g = A.grad;
    g[0 * nasc + p] = cs * acc[1] + ca * gAX[0];
    g[1 * nasc + p] = cs * acc[2] + ca * gAX[1] + ddelta * delta0 * dvtx * vty;
    g[2 * nasc + p] = cs * acc[3];
    g[3 * nasc + p] = -cs * acc[4] - ca * gAY[0] + ddelta * delta0 * vtx * dvty;
    g[4 * nasc + p] = -cs * acc[5] - ca * gAY[1];
    g[5 * nasc + p] = -cs * acc[6];
  }
}

}  // namespace

cudaError_t launch_data(const DataArgs& a, cudaStream_t s) {
  const int64_t nasc = (int64_t)a.L.w * a.L.h;
  const int64_t blocks = (nasc + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks <= 0) return cudaSuccess;
  data_kernel<<<(unsigned)blocks, kWarpsPerBlock * kWarp, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace octmc
