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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace octmc {
namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kOutLanes = 29;
constexpr int kOutPerIter = 4 * kOutLanes;
constexpr unsigned kFull = 0xffffffffu;

struct Vol {
  const void* base;    // the volume; addressed in groups of 4 samples
  unsigned roff[4];    // row offsets (in groups) of the 4 neighbour rows
  unsigned coff[4];    // column offsets (in groups) of the 4 neighbour columns
  float wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
  int q, r;            // floor(dz) = 4 q + r, 0 <= r < 4
  int bx, by;          // floor of the transverse coordinates
};

// Coordinate split of the 6 displacement values of A-scan (i, j) by lanes
// 0..5 (lane = 3 V + c), broadcast to the warp: floor(u) and the float
// fraction for u = i + dx and u = j + dy clamped to [-4, n + 3] (beyond that
// every tap is an edge sample) and u = dz clamped to +-(d + 8) (all depth
// taps are then edge samples).  Integer arithmetic only (split_exact).
__device__ __forceinline__ void split_displacement(const double* disp, int64_t nasc, int64_t p, int i,
                                                   int j, const LevelDev& L, int lane, int base[6],
                                                   float frac[6]) {
  int b = 0;
  float t = 0.f;
  if (lane < 6) {
    const int c = lane % 3;
    const unsigned long long bits =
        (unsigned long long)__double_as_longlong(disp[(int64_t)lane * nasc + p]);
    if (c == 0) split_exact(bits, i, -4, L.w + 3, &b, &t);
    else if (c == 1) split_exact(bits, j, -4, L.h + 3, &b, &t);
    else split_exact(bits, 0, -L.d - 8, L.d + 8, &b, &t);
  }
#pragma unroll
  for (int c = 0; c < 6; c++) {
    base[c] = __shfl_sync(0xffffffffu, b, c);
    frac[c] = __shfl_sync(0xffffffffu, t, c);
  }
}

__device__ __forceinline__ void setup_vol(Vol& V, const void* vol, const LevelDev& L, const int base[3],
                                          const float frac[3]) {
  V.bx = base[0];
  V.by = base[1];
  const int kz0 = base[2];
  V.q = kz0 >> 2;  // arithmetic shift: floor division by 4
  V.r = kz0 & 3;
  keys_weights(frac[0], V.wx, V.dwx);
  keys_weights(frac[1], V.wy, V.dwy);
  keys_weights(frac[2], V.wz, V.dwz);
  const unsigned nq = (unsigned)(L.dp >> 2);
#pragma unroll
  for (int a = 0; a < 4; a++) {
    V.roff[a] = (unsigned)clampi(V.by - 1 + a, L.h) * (unsigned)L.w * nq;
    V.coff[a] = (unsigned)clampi(V.bx - 1 + a, L.w) * nq;
  }
  V.base = vol;
}

// Four consecutive samples (one aligned group) widened to float: float32
// storage is one 16-byte load, bfloat16/float16 one 8-byte load.
template <typename T>
__device__ __forceinline__ float4 load4(const void* base, unsigned idx);
template <>
__device__ __forceinline__ float4 load4<float>(const void* base, unsigned idx) {
  return __ldg(reinterpret_cast<const float4*>(base) + idx);
}
template <>
__device__ __forceinline__ float4 load4<__nv_bfloat16>(const void* base, unsigned idx) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(base) + idx);
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                     __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}
template <>
__device__ __forceinline__ float4 load4<__half>(const void* base, unsigned idx) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(base) + idx);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
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
template <typename S>
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
      const float4 s = load4<S>(V.base, V.roff[b] + V.coff[a] + qc);
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

#ifndef OCTMC_DATA_MINB
#define OCTMC_DATA_MINB 3
#endif
// The whole data-term computation of output A-scan p by one warp.
template <typename T>
__device__ __forceinline__ void data_ascan(const DataArgs& A, int64_t p, int lane) {
  const LevelDev& L = A.L;
  const int64_t nasc = (int64_t)L.w * L.h;
  const int i = (int)(p % L.w), j = (int)(p / L.w);

  int base[6];
  float frac[6];
  split_displacement(A.disp, nasc, p, i, j, L, lane, base, frac);
  Vol VX, VY;
  setup_vol(VX, L.sx, L, base, frac);
  setup_vol(VY, L.sy, L, base + 3, frac + 3);

  const float inv_eps = 1.0f / A.eps_h;
  const bool ssd = (A.loss == OCTMC_LOSS_SSD);
  float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int kb = 0; kb < L.d; kb += kOutPerIter) {
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

  // ---- per-A-scan scalars (Eq. 6-8), float, every lane
  float vtx = 1.f, dvtx = 0.f, vty = 1.f, dvty = 0.f;
  if (L.vx) {  // Eq. 7: X validity along y at j + dy^X (the weights of S^X in y)
    vtx = 0.f;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const float s = L.vx[clampi(VX.by - 1 + b, L.h)];
      vtx = fmaf(VX.wy[b], s, vtx);
      dvtx = fmaf(VX.dwy[b], s, dvtx);
    }
  }
  if (L.vy) {  // Y validity along x at i + dx^Y
    vty = 0.f;
#pragma unroll
    for (int a = 0; a < 4; a++) {
      const float s = L.vy[clampi(VY.bx - 1 + a, L.w)];
      vty = fmaf(VY.wx[a], s, vty);
      dvty = fmaf(VY.dwx[a], s, dvty);
    }
  }
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
  const float eta = (float)A.eta;
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
  if (lane == 0) A.str_out[p] = out;
  else if (lane == 1) A.ang_out[p] = out;
  else if (lane < 8 && A.grad) A.grad[(int64_t)(lane - 2) * nasc + p] = out;
}

template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * kWarp, OCTMC_DATA_MINB)
data_kernel(const DataArgs A) {
  const int64_t p = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (p >= (int64_t)A.L.w * A.L.h) return;  // warp-uniform
  data_ascan<T>(A, p, threadIdx.x & 31);
}

// Several problems ("slots") in one launch: grid (x, slots), block
// (x, s) takes A-scans x*8 .. x*8+7 of slot s (blocks past a slot's end exit
// at once).  The slots' arguments travel in the kernel's parameter block and
// the slot index is uniform per block.  Each A-scan's result does not depend
// on which other slots are in the launch.
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * kWarp, OCTMC_DATA_MINB)
data_multi_kernel(const __grid_constant__ DataMulti M) {
  const DataArgs& A = M.da[blockIdx.y];
  const int64_t p = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (p >= (int64_t)A.L.w * A.L.h) return;  // warp-uniform
  data_ascan<T>(A, p, threadIdx.x & 31);
}

// Motion-corrected resampling and merging of one A-scan (warp): both scans
// resampled along depth at the displaced positions (the derivative parts of
// sample_block are dead code here), merged with the per-A-scan weights.
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * kWarp, OCTMC_DATA_MINB)
resample_merge_kernel(const LevelDev L, const double* __restrict__ disp, const float* __restrict__ weights,
                      float* merged, float* cx, float* cy) {
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
    if (lane >= 1 && lane <= kOutLanes) {
#pragma unroll
      for (int o = 0; o < 4; o++) {
        const int k = kb + 4 * (lane - 1) + o;
        if (k < L.d) {
          const int64_t e = p * L.d + k;
          if (merged) merged[e] = fmaf(wx, IX[o], wy * IY[o]);
          if (cx) cx[e] = IX[o];
          if (cy) cy[e] = IY[o];
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_resample_merge(const LevelDev& L, const double* disp, const float* weights, float* merged,
                                  float* cx, float* cy, cudaStream_t s) {
  const int64_t nasc = (int64_t)L.w * L.h;
  const int64_t blocks = (nasc + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks <= 0) return cudaSuccess;
  if (L.dtype == OCTMC_BF16)
    resample_merge_kernel<__nv_bfloat16><<<(unsigned)blocks, kWarpsPerBlock * kWarp, 0, s>>>(L, disp, weights, merged, cx, cy);
  else if (L.dtype == OCTMC_F16)
    resample_merge_kernel<__half><<<(unsigned)blocks, kWarpsPerBlock * kWarp, 0, s>>>(L, disp, weights, merged, cx, cy);
  else
    resample_merge_kernel<float><<<(unsigned)blocks, kWarpsPerBlock * kWarp, 0, s>>>(L, disp, weights, merged, cx, cy);
  return cudaGetLastError();
}

cudaError_t launch_data_multi(const DataMulti& M, int dtype, cudaStream_t s) {
  if (M.nslots <= 0) return cudaSuccess;
  int64_t most = 0;
  for (int k = 0; k < M.nslots; k++) most = max(most, (int64_t)M.da[k].L.w * M.da[k].L.h);
  const int64_t bx = (most + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (bx <= 0) return cudaSuccess;
  const dim3 g((unsigned)bx, (unsigned)M.nslots);
  if (dtype == OCTMC_BF16)
    data_multi_kernel<__nv_bfloat16><<<g, kWarpsPerBlock * kWarp, 0, s>>>(M);
  else if (dtype == OCTMC_F16)
    data_multi_kernel<__half><<<g, kWarpsPerBlock * kWarp, 0, s>>>(M);
  else
    data_multi_kernel<float><<<g, kWarpsPerBlock * kWarp, 0, s>>>(M);
  return cudaGetLastError();
}

cudaError_t launch_data(const DataArgs& a, cudaStream_t s) {
  const int64_t nasc = (int64_t)a.L.w * a.L.h;
  const int64_t blocks = (nasc + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks <= 0) return cudaSuccess;
  if (a.L.dtype == OCTMC_BF16)
    data_kernel<__nv_bfloat16><<<(unsigned)blocks, kWarpsPerBlock * kWarp, 0, s>>>(a);
  else if (a.L.dtype == OCTMC_F16)
    data_kernel<__half><<<(unsigned)blocks, kWarpsPerBlock * kWarp, 0, s>>>(a);
  else
    data_kernel<float><<<(unsigned)blocks, kWarpsPerBlock * kWarp, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace octmc
