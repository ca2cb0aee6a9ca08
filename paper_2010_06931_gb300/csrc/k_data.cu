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
// Mapping: one warp per output A-scan; a block's 8 warps take a tile of
// 4 x 2 neighbouring A-scans (their 4 x 4 neighbourhoods overlap, which the
// L1 cache turns into hits); 64 registers per thread, so 4 blocks (32 warps)
// per SM keep loads in flight -- the kernel waits on memory latency more
// than on arithmetic.  Depth is processed in blocks of 116
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
#include "sample.cuh"

namespace octmc {
namespace {

#ifndef OCTMC_DATA_MINB
#define OCTMC_DATA_MINB 4
#endif
// The data-term computation of output A-scan p by one warp (base and frac:
// the coordinate split of its 6 displacement values).
template <typename T>
__device__ __forceinline__ void data_core(const DataArgs& A, int64_t p, int lane, const int base[6],
                                          const float frac[6]) {
  const LevelDev& L = A.L;
  const int64_t nasc = (int64_t)L.w * L.h;
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

#ifndef OCTMC_DTILE_X
#define OCTMC_DTILE_X 4
#endif
constexpr int kDTileX = OCTMC_DTILE_X;  // direct kernel: a block's 8 A-scans as kDTileX x (8 / kDTileX)
constexpr int kDTileY = kWarpsPerBlock / kDTileX;

// A-scan of warp `warp` of direct block b: tiles of kDTileX x kDTileY.
__device__ __forceinline__ int64_t direct_ascan(const LevelDev& L, int b, int warp) {
  const int tiles_x = (L.w + kDTileX - 1) / kDTileX;
  const int i = (b % tiles_x) * kDTileX + warp % kDTileX, j = (b / tiles_x) * kDTileY + warp / kDTileX;
  return (i < L.w && j < L.h) ? (int64_t)j * L.w + i : -1;
}

__host__ __device__ inline int64_t direct_blocks(int w, int h) {
  return (int64_t)((w + kDTileX - 1) / kDTileX) * ((h + kDTileY - 1) / kDTileY);
}

template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * kWarp, OCTMC_DATA_MINB)
data_kernel(const DataArgs A) {
  const int64_t p = direct_ascan(A.L, blockIdx.x, threadIdx.x >> 5);
  if (p < 0) return;  // warp-uniform
  data_ascan<T>(A, p, threadIdx.x & 31);
}

// Several problems ("slots") in one launch: grid (x, slots), block
// (x, s) takes tile x of slot s (blocks past a slot's last tile exit at
// once).  The slots' arguments travel in the kernel's parameter block and
// the slot index is uniform per block.  Each A-scan's result does not depend
// on which other slots are in the launch.
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * kWarp, OCTMC_DATA_MINB)
data_multi_kernel(const __grid_constant__ DataMulti M) {
  const DataArgs& A = M.da[blockIdx.y];
  if ((int64_t)blockIdx.x >= direct_blocks(A.L.w, A.L.h)) return;
  const int64_t p = direct_ascan(A.L, blockIdx.x, threadIdx.x >> 5);
  if (p < 0) return;  // warp-uniform
  data_ascan<T>(A, p, threadIdx.x & 31);
}

}  // namespace

cudaError_t launch_data_multi(const DataMulti& M, int dtype, cudaStream_t s) {
  if (M.nslots <= 0) return cudaSuccess;
  int64_t bx = 0;
  for (int k = 0; k < M.nslots; k++) bx = max(bx, direct_blocks(M.da[k].L.w, M.da[k].L.h));
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
  const int64_t blocks = direct_blocks(a.L.w, a.L.h);
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
