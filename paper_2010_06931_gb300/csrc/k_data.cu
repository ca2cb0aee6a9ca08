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
#include "data.cuh"
#include "sample.cuh"

namespace octmc {
namespace {

#ifndef OCTMC_DATA_MINB
#define OCTMC_DATA_MINB 4
#endif
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
