// Data-term evaluation that allocates nothing: octmc_data_term_static.
//
// For callers that cannot call cudaMalloc -- code running inside a memory
// pool or allocator callback, under a framework that owns all device
// memory, or on a path where allocation is forbidden after start-up -- this
// entry point evaluates the data term (S^str, S^ang and their gradient) of
// one grid directly on caller-owned device buffers.  Its scratch (the
// per-A-scan partial sums, the float gradient, block partials and a
// completion counter) lives in one file-scope __device__ array of fixed
// size, which every GPU that loads the library holds until the process
// exits.  The array's host-side name is not a device address: its device
// address is looked up with cudaGetSymbolAddress, for the current device,
// on every call, and passed to the kernels.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "common.cuh"

namespace octmc {
namespace {

constexpr int64_t kStaticMaxAscans = int64_t(1) << 18;  // 262,144 A-scans, e.g. 512 x 512
constexpr int kFinishBlocks = 152;
constexpr int kFinishThreads = 256;

struct StaticScratch {
  float str[kStaticMaxAscans];
  float ang[kStaticMaxAscans];
  float grad[6 * kStaticMaxAscans];
  double partials[2 * kFinishBlocks];
  unsigned counter;
};

// 8 MiB (+ 2.4 KiB) per device.
__device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticScratch)];

// Widens the float gradient into the caller's float64 buffer and adds the
// per-A-scan data sums in a fixed order (block trees, last block adds the
// block partials); sums_out[0] = S^str, sums_out[1] = S^ang.
__global__ void __launch_bounds__(kFinishThreads) static_finish_kernel(StaticScratch* s, int64_t n,
                                                                       double* grad_out, double* sums_out) {
  __shared__ double sm[2][kFinishThreads / 32];
  __shared__ bool is_last;
  double v0 = 0.0, v1 = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * kFinishThreads + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * kFinishThreads) {
    v0 += widen_exact(s->str[p]);
    v1 += widen_exact(s->ang[p]);
    if (grad_out)
#pragma unroll
      for (int c = 0; c < 6; c++) grad_out[c * n + p] = widen_exact(s->grad[c * n + p]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  if (lane == 0) {
    sm[0][warp] = v0;
    sm[1][warp] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kFinishThreads / 32; w++) {
      a += sm[0][w];
      b += sm[1][w];
    }
    s->partials[2 * blockIdx.x] = a;
    s->partials[2 * blockIdx.x + 1] = b;
    __threadfence();
    is_last = (atomicAdd(&s->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    double a = 0.0, b = 0.0;
    for (unsigned k = 0; k < gridDim.x; k++) {
      a += s->partials[2 * k];
      b += s->partials[2 * k + 1];
    }
    sums_out[0] = a;
    sums_out[1] = b;
    s->counter = 0u;
  }
}

// Device address of the scratch array for the current device.  It is looked
// up on every call (cudaGetSymbolAddress allocates nothing and is cheap), so
// there is no per-device cache to race on between host threads and no stale
// address after the caller resets the device.
cudaError_t scratch_for_current_device(StaticScratch** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<StaticScratch*>(ptr);
  return cudaSuccess;
}

}  // namespace
}  // namespace octmc

using namespace octmc;

extern "C" int octmc_data_term_static(const float* sx, const float* sy, const float* ax, const float* ay,
                                      const float* vx, const float* vy, int w, int h, int d,
                                      const double* disp, double eta, double delta0, double eps_h, int loss,
                                      double* grad_out, double* sums_out, void* stream) {
  if (!sx || !sy || !disp || !sums_out || w < 1 || h < 1 || d < 4 || (d & 3) != 0)
    return OCTMC_ERR_INVALID_ARG;
  if ((ax == nullptr) != (ay == nullptr)) return OCTMC_ERR_INVALID_ARG;
  // the kernel reads the volumes in aligned 16-byte groups of 4 samples
  if ((reinterpret_cast<uintptr_t>(sx) & 15u) || (reinterpret_cast<uintptr_t>(sy) & 15u)) return OCTMC_ERR_INVALID_ARG;
  if (!(eta > 0) || !(eps_h > 0) || !(delta0 >= 0) || !std::isfinite(eta) || !std::isfinite(eps_h) ||
      !std::isfinite(delta0))
    return OCTMC_ERR_INVALID_ARG;
  if (loss != OCTMC_LOSS_PSEUDO_HUBER && loss != OCTMC_LOSS_SSD) return OCTMC_ERR_INVALID_ARG;
  const int64_t n = (int64_t)w * h;
  if (n > kStaticMaxAscans) return OCTMC_ERR_SCRATCH_LIMIT;
  // the data kernel addresses a volume in 32-bit units of 4 samples
  if (n * (d / 4) >= (int64_t)1 << 32) return OCTMC_ERR_INVALID_ARG;
  const cudaStream_t st = (cudaStream_t)stream;
  StaticScratch* s = nullptr;
  if (scratch_for_current_device(&s) != cudaSuccess) {
    cudaGetLastError();
    return OCTMC_ERR_CUDA;
  }
  // the completion counter must start at zero whatever the last call left
  if (cudaMemsetAsync(&s->counter, 0, sizeof(unsigned), st) != cudaSuccess) {
    cudaGetLastError();
    return OCTMC_ERR_CUDA;
  }
  DataArgs A;
  std::memset(&A, 0, sizeof(A));
  A.L.w = w;
  A.L.h = h;
  A.L.d = d;
  A.L.dp = d;  // d is a multiple of 4: the caller's [h][w][d] is the kernel's layout
  A.L.sx = const_cast<float*>(sx);
  A.L.sy = const_cast<float*>(sy);
  A.L.ax = const_cast<float*>(ax);
  A.L.ay = const_cast<float*>(ay);
  A.L.vx = const_cast<float*>(vx);
  A.L.vy = const_cast<float*>(vy);
  A.disp = disp;
  A.str_out = s->str;
  A.ang_out = s->ang;
  A.grad = grad_out ? s->grad : nullptr;
  A.eta = eta;
  A.delta0 = ax ? delta0 : 0.0;
  A.eps_h = (float)eps_h;
  A.loss = loss;
  if (launch_data(A, st) != cudaSuccess) {
    cudaGetLastError();
    return OCTMC_ERR_CUDA;
  }
  static_finish_kernel<<<kFinishBlocks, kFinishThreads, 0, st>>>(s, n, grad_out, sums_out);
  if (cudaGetLastError() != cudaSuccess) return OCTMC_ERR_CUDA;
  return OCTMC_OK;
}
