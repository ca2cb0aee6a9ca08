// History update and compact-form L-BFGS algebra of the device-resident
// level solve (Ploner et al., Sec. 2.1; Byrd, Nocedal & Schnabel compact
// representation), shared by the products kernel and the persistent
// small-level kernel.  Each block that runs it works on its own copy of the
// SolveState.
#pragma once
#include <math.h>

#include "common.cuh"

namespace octmc {
namespace {

// ---- the compact-form algebra (one thread), after the products are known

__device__ __forceinline__ double& SYa(SolveState* S, int a, int b) { return S->SY[a * (kMaxM + 1) + b]; }
__device__ __forceinline__ double& YYa(SolveState* S, int a, int b) { return S->YY[a * (kMaxM + 1) + b]; }

__device__ void history_update(SolveState* S) {
  const double* r = S->dots;
  const int K = 2 * S->ncand;
  const int nb = S->spare;
  if (S->mode == kModeAccept) {
    const int t_new = S->k;  // the new pair is the last candidate
    const double s_y = r[2 * (2 * t_new)], y_y = r[2 * K];
    if (s_y > 1e-12 * y_y && isfinite(s_y) && isfinite(y_y)) {
      for (int t = 0; t < S->k; t++) {
        const int b = S->order[t];
        SYa(S, b, nb) = r[2 * (2 * t)];
        const double v = r[2 * (2 * t + 1)];
        YYa(S, b, nb) = v;
        YYa(S, nb, b) = v;
      }
      SYa(S, nb, nb) = s_y;
      YYa(S, nb, nb) = y_y;
      if (S->k == S->m) {
        for (int t = 0; t + 1 < S->k; t++) S->order[t] = S->order[t + 1];
        S->k--;
      }
      S->order[S->k++] = nb;
      // the spare buffer: the first id not in the history
      int fb = 0;
      for (int b = 0; b <= S->m; b++) {
        bool used = false;
        for (int t = 0; t < S->k; t++) used |= (S->order[t] == b);
        if (!used) {
          fb = b;
          break;
        }
      }
      S->spare = fb;
    }
  }
  for (int t = 0; t < S->ncand; t++) {
    S->sg[S->cand[t]] = r[2 * (2 * t) + 1];
    S->yg[S->cand[t]] = r[2 * (2 * t + 1) + 1];
  }
  S->gg = r[2 * K + 1];
}

// Block-wide copy of the solver state, 16 bytes per load, all of a thread's
// loads issued before its stores.
template <int kBlock>
__device__ __forceinline__ void copy_state(SolveState* dst, const SolveState* src) {
  constexpr int kWords = (int)(sizeof(SolveState) / 16);
  constexpr int kPer = (kWords + kBlock - 1) / kBlock;
  const int4* s4 = reinterpret_cast<const int4*>(src);
  int4* d4 = reinterpret_cast<int4*>(dst);
  int4 buf[kPer];
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    const int w = threadIdx.x + i * kBlock;
    if (w < kWords) buf[i] = s4[w];
  }
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    const int w = threadIdx.x + i * kBlock;
    if (w < kWords) d4[w] = buf[i];
  }
}
static_assert(sizeof(SolveState) % 16 == 0, "solver state is copied in 16-byte words");

// After the products: history update and the compact-form
// (Byrd, Nocedal & Schnabel) direction dir = -H g with H0 = gamma I, gamma
// from the newest pair, as coefficients of g and the history vectors; g . dir
// follows from the products (no extra pass).  Run by every thread of one
// block: the k x k blocks of S'Y and Y'Y are staged in shared memory, the
// matrix-vector rows are spread over threads, the two triangular solves run
// in one thread; every sum keeps the serial order, so the result does not
// depend on the thread count.
struct Algebra {
  double R[kMaxM][kMaxM];   // R_ij = s_i . y_j
  double YY[kMaxM][kMaxM];  // y_i . y_j
  double a[kMaxM], b[kMaxM], u[kMaxM], w[kMaxM], top[kMaxM];
  double rd[kMaxM];         // 1 / R_ii
};

__device__ void after_products(SolveState* S, Algebra& A) {
  if (threadIdx.x == 0) history_update(S);
  __syncthreads();
  const int k = S->k;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t / k, j = t % k;
    A.R[i][j] = SYa(S, S->order[i], S->order[j]);
    A.YY[i][j] = YYa(S, S->order[i], S->order[j]);
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    A.a[i] = S->sg[S->order[i]];
    A.b[i] = S->yg[S->order[i]];
    // the divisions (long float64 sequences) off the serial solves below
    A.rd[i] = 1.0 / SYa(S, S->order[i], S->order[i]);
  }
  __syncthreads();
  double gamma = 0.0;
  if (k > 0) gamma = A.R[k - 1][k - 1] / A.YY[k - 1][k - 1];
  if (k > 0 && threadIdx.x == 0) {  // u = R^{-1} a (R upper triangular)
    for (int i = k - 1; i >= 0; i--) {
      double s = A.a[i];
      for (int j = i + 1; j < k; j++) s -= A.R[i][j] * A.u[j];
      A.u[i] = s * A.rd[i];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {  // w = (D + gamma Y'Y) u - gamma b
    double s = A.R[i][i] * A.u[i];
    for (int j = 0; j < k; j++) s += gamma * A.YY[i][j] * A.u[j];
    A.w[i] = s - gamma * A.b[i];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double gd;
  if (k > 0) {
    for (int i = 0; i < k; i++) {  // top = R^{-T} w
      double s = A.w[i];
      for (int j = 0; j < i; j++) s -= A.R[j][i] * A.top[j];
      A.top[i] = s * A.rd[i];
    }
    S->cg = -gamma;
    S->nc = 0;
    gd = -gamma * S->gg;
    for (int i = 0; i < k; i++) {
      S->hid[S->nc] = 2 * S->order[i];
      S->coef[S->nc++] = -A.top[i];
      S->hid[S->nc] = 2 * S->order[i] + 1;
      S->coef[S->nc++] = gamma * A.u[i];
      gd += -A.top[i] * A.a[i] + gamma * A.u[i] * A.b[i];
    }
    if (!(gd < 0.0)) {  // not a descent direction: drop the history, -g
      S->k = 0;
      S->cg = -1.0;
      S->nc = 0;
      gd = -S->gg;
    }
  } else {
    S->cg = -1.0;
    S->nc = 0;
    gd = -S->gg;
  }
  S->dg0 = gd;
  S->a = (S->k == 0) ? 1.0 / sqrt(S->gg) : 1.0;
  S->lo = 0.0;
  S->hi = INFINITY;
  S->have_lo = 0;
  S->ls = 0;
  S->mode = kModeTrial;
}

}  // namespace
}  // namespace octmc
