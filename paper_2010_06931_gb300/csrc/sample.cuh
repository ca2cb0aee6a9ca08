// Displaced Catmull-Rom sampling of one A-scan by one warp, shared by the
// data-term kernel and the final resampling (Ploner et al., Eq. 2 and
// Sec. 2.1): coordinate split, per-volume setup, the lane-parallel
// transverse 4x4 interpolation of aligned groups of 4 input samples and the
// 4-tap axial filter with its halo shuffles.
//
// Depth is processed in blocks of 116 outputs; lane L (1..29) owns outputs
// kb + 4(L-1) .. +3, loads one aligned group of 4 input samples from each of
// the 16 transverse neighbour columns with one 128-bit load per column
// (coalesced along depth across the warp), and gets the neighbouring input
// depths the axial filter needs from the adjacent lanes by shuffles.  Lanes
// 0, 30 and 31 only supply those halo values.
#pragma once
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

// ---------------------------------------------------------------- packed float pairs
// Two float lanes per instruction (fma.rn.f32x2): each half is rounded like
// fmaf, so packed and scalar code give bitwise equal results; the packed
// form halves the issue slots of the interpolation's multiply-adds.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// Four consecutive depth samples as two packed pairs (k, k+1), (k+2, k+3).
struct Q4 {
  float2 lo, hi;
};

__device__ __forceinline__ Q4 q4(const float4& v) { return {make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ Q4 q4zero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

// acc += w * s on all four samples (w broadcast to both halves)
__device__ __forceinline__ void qfma(Q4& acc, float2 w, const Q4& s) {
  acc.lo = ffma2(w, s.lo, acc.lo);
  acc.hi = ffma2(w, s.hi, acc.hi);
}

__device__ __forceinline__ float4 f4(const Q4& q) { return make_float4(q.lo.x, q.lo.y, q.hi.x, q.hi.y); }

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
#ifndef OCTMC_AXIAL_PACKED
#define OCTMC_AXIAL_PACKED 1
#endif
#if OCTMC_AXIAL_PACKED
  // outputs in packed pairs (o, o + 1); each half adds its 4 taps in the
  // scalar order
#pragma unroll
  for (int o = 0; o < 4; o += 2) {
    float2 a = make_float2(0.f, 0.f), az = a, ax = a, ay = a;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const float2 w = make_float2(wz[c], wz[c]), dw = make_float2(dwz[c], dwz[c]);
      const float2 ev = make_float2(e[R + o + c], e[R + o + 1 + c]);
      a = ffma2(w, ev, a);
      az = ffma2(dw, ev, az);
      ax = ffma2(w, make_float2(ex[R + o + c], ex[R + o + 1 + c]), ax);
      ay = ffma2(w, make_float2(ey[R + o + c], ey[R + o + 1 + c]), ay);
    }
    I[o] = a.x; I[o + 1] = a.y;
    Iz[o] = az.x; Iz[o + 1] = az.y;
    Ix[o] = ax.x; Ix[o + 1] = ax.y;
    Iy[o] = ay.x; Iy[o + 1] = ay.y;
  }
#else
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
#endif
}

// Interpolated values (and their displacement derivatives) of one volume
// at the lane's 4 outputs.  qk: first input depth of the lane's group
// (samples, may lie outside the volume); qc: index of that group's (clamped)
// samples in the volume.
template <typename S>
__device__ __forceinline__ void sample_group(const Vol& V, int qk, unsigned qc, int dp, float I[4], float Iz[4],
                                             float Ix[4], float Iy[4]) {
  // transverse 4 x 4 interpolation of the group and its x / y derivatives,
  // in packed pairs along depth (same operations and order as scalar FMAs)
  Q4 Tq = q4zero(), Txq = q4zero(), Tyq = q4zero();
#pragma unroll
  for (int b = 0; b < 4; b++) {
    Q4 U = q4zero(), Ux = q4zero();
#pragma unroll
    for (int a = 0; a < 4; a++) {
      const unsigned idx = V.roff[b] + V.coff[a] + qc;
      const Q4 s = q4(load4<S>(V.base, idx));
      qfma(U, make_float2(V.wx[a], V.wx[a]), s);
      qfma(Ux, make_float2(V.dwx[a], V.dwx[a]), s);
    }
    qfma(Tq, make_float2(V.wy[b], V.wy[b]), U);
    qfma(Txq, make_float2(V.wy[b], V.wy[b]), Ux);
    qfma(Tyq, make_float2(V.dwy[b], V.dwy[b]), U);
  }
  float4 T = f4(Tq), Tx = f4(Txq), Ty = f4(Tyq);
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

// Interpolated values (and their displacement derivatives) of one volume
// at the lane's 4 outputs of the depth block starting at kb, from the
// volume in global memory.
template <typename S>
__device__ __forceinline__ void sample_block(const Vol& V, int kb, int lane, int dp, float I[4],
                                             float Iz[4], float Ix[4], float Iy[4]) {
  const int qk = kb + 4 * V.q + 4 * (lane - 1);  // first input depth of the lane's group
  const unsigned qc = (unsigned)(min(max(qk, 0), dp - 4) >> 2);
  sample_group<S>(V, qk, qc, dp, I, Iz, Ix, Iy);
}

}  // namespace
}  // namespace octmc
