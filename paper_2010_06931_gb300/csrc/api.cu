// Host side of liboctmc: the problem object (device pyramid and chains), one
// objective evaluation, eta, the on-device L-BFGS and the level / full
// solves, behind the C ABI declared in include/octmc.h.
//
// All vectors of the optimiser (displacements, gradients, directions, the
// L-BFGS history, all float64) live in device memory; the host only reads the
// few scalars the line search and the compact L-BFGS algebra need (f,
// grad . dir, and at most 4m+7 dot products per iteration).
#include <algorithm>
#include <cstddef>
#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"

using namespace octmc;

namespace {

struct CudaFail {
  int code;
};

#define CK(call)                                                       \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      throw CudaFail{e_ == cudaErrorMemoryAllocation ? OCTMC_ERR_OOM   \
                                                     : OCTMC_ERR_CUDA}; \
    }                                                                  \
  } while (0)

template <typename T>
T* dalloc(size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw CudaFail{e == cudaErrorMemoryAllocation ? OCTMC_ERR_OOM : OCTMC_ERR_CUDA};
  }
  return static_cast<T*>(p);
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

int half_up(int n) { return (n + 1) / 2; }
int pad4(int d) { return (d + 3) & ~3; }

// Time-ordered chain of the A-scans of one volume: prev/next neighbour in
// acquisition order and the weight dt_min / dt of each pair (ties weigh 1).
void build_chain(const std::vector<double>& t, std::vector<int>& prev, std::vector<int>& next,
                 std::vector<float>& wprev, std::vector<float>& wnext) {
  const int n = (int)t.size();
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return t[a] < t[b] || (t[a] == t[b] && a < b); });
  double dtmin = std::numeric_limits<double>::infinity();
  for (int m = 0; m + 1 < n; m++) {
    const double dt = t[order[m + 1]] - t[order[m]];
    if (dt > 0 && dt < dtmin) dtmin = dt;
  }
  prev.assign(n, -1);
  next.assign(n, -1);
  wprev.assign(n, 0.f);
  wnext.assign(n, 0.f);
  for (int m = 0; m + 1 < n; m++) {
    const int a = order[m], b = order[m + 1];
    const double dt = t[b] - t[a];
    const double om = std::isinf(dtmin) ? 1.0 : dtmin / std::max(dt, dtmin);
    next[a] = b;
    wnext[a] = (float)om;
    prev[b] = a;
    wprev[b] = (float)om;
  }
}

std::vector<double> time_down(const std::vector<double>& t, int w, int h) {
  const int w2 = half_up(w), h2 = half_up(h);
  std::vector<double> o((size_t)w2 * h2);
  for (int j = 0; j < h2; j++)
    for (int i = 0; i < w2; i++) {
      const int i1 = std::min(2 * i + 1, w - 1), j1 = std::min(2 * j + 1, h - 1);
      o[(size_t)j * w2 + i] = (t[(size_t)2 * j * w + 2 * i] + t[(size_t)2 * j * w + i1] +
                               t[(size_t)j1 * w + 2 * i] + t[(size_t)j1 * w + i1]) /
                              4.0;
    }
  return o;
}

}  // namespace

// ====================================================================== L-BFGS
struct octmc_lbfgs {
  int64_t n = 0;
  int m = 0;
  cudaStream_t st = nullptr;
  std::vector<double*> S, Y;  // m + 1 buffers each
  std::vector<int> order;     // stored pairs, oldest first (buffer ids)
  int spare = 0;              // buffer receiving the next pair
  std::vector<double> SY, YY; // (m+1)^2, indexed by buffer ids
  double* partials = nullptr;
  unsigned* counter = nullptr;
  double* dots_dev = nullptr;
  double* dots_host = nullptr; // pinned, hist_dots_outputs(2 (m + 1))
  // results of the last prepare(): per stored buffer s.g and y.g, g.g, max|g|
  std::vector<double> sg, yg;
  double gg = 0.0, gmax = 0.0;

  ~octmc_lbfgs() {
    for (double* p : S) dfree(p);
    for (double* p : Y) dfree(p);
    dfree(partials);
    dfree(counter);
    dfree(dots_dev);
    if (dots_host) cudaFreeHost(dots_host);
  }

  void init(int64_t n_, int m_, cudaStream_t s) {
    n = n_;
    m = m_;
    st = s;
    S.assign(m + 1, nullptr);
    Y.assign(m + 1, nullptr);
    for (int b = 0; b <= m; b++) {
      S[b] = dalloc<double>((size_t)n);
      Y[b] = dalloc<double>((size_t)n);
    }
    SY.assign((size_t)(m + 1) * (m + 1), 0.0);
    YY.assign((size_t)(m + 1) * (m + 1), 0.0);
    sg.assign(m + 1, 0.0);
    yg.assign(m + 1, 0.0);
    const int nout = hist_dots_outputs(2 * (m + 1));
    partials = dalloc<double>((size_t)nout * hist_dots_blocks(n));
    counter = dalloc<unsigned>(1);
    CK(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    dots_dev = dalloc<double>(nout);
    CK(cudaMallocHost(&dots_host, sizeof(double) * nout));
    reset();
  }

  void reset() {
    order.clear();
    spare = 0;
  }
  int k() const { return (int)order.size(); }
  double& sy(int a, int b) { return SY[(size_t)a * (m + 1) + b]; }
  double& yy(int a, int b) { return YY[(size_t)a * (m + 1) + b]; }

  int free_buffer() const {
    for (int b = 0; b <= m; b++)
      if (std::find(order.begin(), order.end(), b) == order.end()) return b;
    return 0;
  }

  // One pass over the history: if new_pair, the pair in buffer `spare` is
  // tested (s'y > 1e-12 y'y) and appended (dropping the oldest when full);
  // if g != null, s.g and y.g for every stored pair plus g.g and max|g| are
  // taken for the next direction.  launch_prepare enqueues the dot products
  // (the stored pairs and the new one against the probes y_new and g) and
  // their copy to pinned host memory; finish_prepare (after the stream has
  // synchronised) updates the history.  It returns 1 if a new pair was
  // rejected.
  bool pend_new = false, pend_g = false;
  int pend_K = 0;
  std::vector<int> pend_cand;  // buffers of the history vectors, in order

  void launch_prepare(const double* g, bool new_pair) {
    HistDots hd{};
    int K = 0;
    const int nb = spare;
    pend_cand = order;
    if (new_pair) pend_cand.push_back(nb);
    for (int b : pend_cand) {
      hd.h[K++] = S[b];
      hd.h[K++] = Y[b];
    }
    hd.K = K;
    hd.q0 = new_pair ? Y[nb] : nullptr;
    hd.q1 = g;
    pend_K = K;
    pend_new = new_pair;
    pend_g = (g != nullptr);
    CK(launch_hist_dots(hd, n, partials, counter, dots_dev, st));
    CK(cudaMemcpyAsync(dots_host, dots_dev, sizeof(double) * hist_dots_outputs(K), cudaMemcpyDeviceToHost, st));
  }

  // Output layout of hist_dots for history vector 2t (S of pend_cand[t]) and
  // 2t+1 (Y of pend_cand[t]): [2v] = v . y_new, [2v+1] = v . g.
  int finish_prepare() {
    const double* r = dots_host;
    const int nb = spare, K = pend_K;
    const int t_new = (int)order.size();  // the new pair's slot in pend_cand
    int rejected = 0;
    if (pend_new) {
      const double s_y = r[2 * (2 * t_new)], y_y = r[2 * K];
      if (s_y > 1e-12 * y_y && std::isfinite(s_y) && std::isfinite(y_y)) {
        for (size_t t = 0; t < order.size(); t++) {
          sy(order[t], nb) = r[2 * (2 * t)];
          const double v = r[2 * (2 * t + 1)];
          yy(order[t], nb) = v;
          yy(nb, order[t]) = v;
        }
        sy(nb, nb) = s_y;
        yy(nb, nb) = y_y;
        if ((int)order.size() == m) order.erase(order.begin());
        order.push_back(nb);
        spare = free_buffer();
      } else {
        rejected = 1;
      }
    }
    if (pend_g) {
      for (size_t t = 0; t < pend_cand.size(); t++) {
        sg[pend_cand[t]] = r[2 * (2 * t) + 1];
        yg[pend_cand[t]] = r[2 * (2 * t + 1) + 1];
      }
      gg = r[2 * K + 1];
      gmax = r[2 * K + 2];
    }
    pend_new = pend_g = false;
    return rejected;
  }

  // Drops a launched prepare whose results are not wanted (the history is
  // untouched until finish_prepare).
  void cancel_prepare() { pend_new = pend_g = false; }

  int prepare(const double* g, bool new_pair) {
    launch_prepare(g, new_pair);
    CK(cudaStreamSynchronize(st));
    return finish_prepare();
  }

  // dir = -H g (compact form of Byrd, Nocedal & Schnabel with H0 = gamma I),
  // using the s.g / y.g of the last prepare(g).  Returns g . dir; when that
  // is not negative the history is dropped and dir = -g.
  double direction(const double* g, double* dir) {
    const int k = this->k();
    HistComb lc{};
    double gd;
    if (k > 0) {
      const int last = order[k - 1];
      const double gamma = sy(last, last) / yy(last, last);
      std::vector<double> a(k), b(k), u(k), wv(k), top(k);
      for (int i = 0; i < k; i++) {
        a[i] = sg[order[i]];
        b[i] = yg[order[i]];
      }
      // u = R^{-1} a, R_ij = s_i . y_j (i <= j)
      for (int i = k - 1; i >= 0; i--) {
        double s = a[i];
        for (int j = i + 1; j < k; j++) s -= sy(order[i], order[j]) * u[j];
        u[i] = s / sy(order[i], order[i]);
      }
      // w = (D + gamma Y'Y) u - gamma b
      for (int i = 0; i < k; i++) {
        double s = sy(order[i], order[i]) * u[i];
        for (int j = 0; j < k; j++) s += gamma * yy(order[i], order[j]) * u[j];
        wv[i] = s - gamma * b[i];
      }
      // top = R^{-T} w
      for (int i = 0; i < k; i++) {
        double s = wv[i];
        for (int j = 0; j < i; j++) s -= sy(order[j], order[i]) * top[j];
        top[i] = s / sy(order[i], order[i]);
      }
      lc.g = g;
      lc.cg = -gamma;
      lc.K = 0;
      gd = -gamma * gg;
      for (int i = 0; i < k; i++) {
        lc.h[lc.K] = S[order[i]];
        lc.c[lc.K++] = -top[i];
        lc.h[lc.K] = Y[order[i]];
        lc.c[lc.K++] = gamma * u[i];
        gd += -top[i] * a[i] + gamma * u[i] * b[i];
      }
      if (!(gd < 0.0)) k_reset_steepest(lc, g, gd);
    } else {
      k_reset_steepest(lc, g, gd);
    }
    CK(launch_hist_comb(lc, n, dir, st));
    return gd;
  }

  void k_reset_steepest(HistComb& lc, const double* g, double& gd) {
    reset();
    lc.g = g;
    lc.cg = -1.0;
    lc.K = 0;
    gd = -gg;
  }
};

// ====================================================================== problem
struct Level {
  LevelDev dev{};
  double eta = 1.0;
  double mu = 0.0;
};

struct octmc_problem {
  octmc_desc desc{};
  cudaStream_t st = nullptr;
  bool have_ang = false;
  std::vector<Level> lv;
  // evaluation workspace (sized for level 0)
  float* str = nullptr;
  float* ang = nullptr;
  float* gdata = nullptr;  // data-term gradient (float), consumed by reg_kernel
  double* partials = nullptr;
  unsigned* counters = nullptr;  // [0] msum, [1] reg
  EvalResult* res = nullptr;
  EvalResult* res_host = nullptr;  // pinned
  // solver workspace (level-0 sized, allocated on first solve)
  double* x = nullptr;
  double* g = nullptr;
  double* xt = nullptr;
  double* gt = nullptr;
  double* xb = nullptr;
  double* gb = nullptr;
  double* dir = nullptr;
  octmc_lbfgs* opt = nullptr;
  // device-resident level solve: its state (device + pinned host copy), the
  // product partials, and the capture streams and fork/join events of its graphs
  SolveState* sstate = nullptr;
  LevelStatsDev* lstats = nullptr;       // per solved level, on the device
  LevelStatsDev* lstats_host = nullptr;  // pinned copy
  std::map<int, std::pair<cudaGraph_t, cudaGraphExec_t>> graphs;  // solve graphs by (first, last) level
  double* spartials = nullptr;
  unsigned* scounter = nullptr;
  // the persistent small-level kernel (when persistent_ascans > 0)
  double* lpart = nullptr;
  unsigned* lbar = nullptr;  // [2] grid-barrier state, then [2] the error word (as int)
  int lgrid = 0;
  cudaStream_t cap = nullptr, cap_side = nullptr;
  cudaEvent_t cap_fork = nullptr, cap_join = nullptr;
  unsigned long long* mcounts = nullptr;  // merge: fixed-point density maps [2][h][w]
  // prealignment: induced field and its gradient (level-0 sized), and
  // [T, g . dir] on the device and its pinned host copy
  double* pre_D = nullptr;
  double* pre_G = nullptr;
  double* pre_aux = nullptr;
  double* pre_aux_host = nullptr;
  double* pre_prm = nullptr;  // 2 (w + h) of level 0: parameter gradient scratch / coarse copy
  std::vector<void*> temps;  // float32 pyramid copies while building 16-bit storage
  // optional CUDA-event timing of the data-term kernel (octmc_profile_*)
  bool profile = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double prof_ms = 0.0;
  long long prof_count = 0;
  bool prof_pending = false;

  ~octmc_problem() {
    for (void* t : temps) dfree(t);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (Level& L : lv) {
      LevelDev& d = L.dev;
      dfree(d.sx); dfree(d.sy); dfree(d.ax); dfree(d.ay); dfree(d.vx); dfree(d.vy);
      for (int V = 0; V < 2; V++) {
        dfree(d.prev[V]); dfree(d.next[V]); dfree(d.wprev[V]); dfree(d.wnext[V]);
      }
    }
    dfree(str); dfree(ang); dfree(gdata); dfree(partials); dfree(counters); dfree(res);
    if (res_host) cudaFreeHost(res_host);
    dfree(x); dfree(g); dfree(xt); dfree(gt); dfree(xb); dfree(gb); dfree(dir);
    dfree(mcounts);
    dfree(pre_D); dfree(pre_G); dfree(pre_aux); dfree(pre_prm);
    if (pre_aux_host) cudaFreeHost(pre_aux_host);
    delete opt;
    for (auto& kv : graphs) {
      cudaGraphExecDestroy(kv.second.second);
      cudaGraphDestroy(kv.second.first);
    }
    dfree(sstate);
    dfree(lstats);
    dfree(spartials);
    dfree(scounter);
    dfree(lpart);
    dfree(lbar);
    if (lstats_host) cudaFreeHost(lstats_host);
    if (cap) cudaStreamDestroy(cap);
    if (cap_side) cudaStreamDestroy(cap_side);
    if (cap_fork) cudaEventDestroy(cap_fork);
    if (cap_join) cudaEventDestroy(cap_join);
  }

  int64_t plane(int l) const { return (int64_t)lv[l].dev.w * lv[l].dev.h; }
};

namespace {

void check_device() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  if (!(prop.major == 10 && prop.minor == 3)) throw CudaFail{OCTMC_ERR_UNSUPPORTED};
}

void upload_volume(octmc_problem* P, const float* src, float* dst, int w, int h, int d, int dp) {
  const cudaMemcpyKind kind = P->desc.inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const int64_t cols = (int64_t)w * h;
  // rows of d samples into rows of dp; cudaMemcpy2D limits the row count to
  // what a size_t height takes, so copy in slabs of columns
  const int64_t slab = 1 << 20;
  for (int64_t c0 = 0; c0 < cols; c0 += slab) {
    const int64_t nc = std::min(slab, cols - c0);
    CK(cudaMemcpy2DAsync(dst + c0 * dp, sizeof(float) * dp, src + c0 * d, sizeof(float) * d,
                         sizeof(float) * d, (size_t)nc, kind, P->st));
  }
  CK(launch_pad_depth(dst, cols, d, dp, P->st));
}

template <typename T>
void upload(octmc_problem* P, const T* src, T* dst, size_t count) {
  const cudaMemcpyKind kind = P->desc.inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(dst, src, sizeof(T) * count, kind, P->st));
}

template <typename T>
void upload_host(octmc_problem* P, const std::vector<T>& v, T* dst) {
  CK(cudaMemcpyAsync(dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, P->st));
}

std::vector<double> fetch_times(octmc_problem* P, const double* t, size_t n) {
  std::vector<double> out(n);
  if (P->desc.inputs_on_device) {
    CK(cudaMemcpyAsync(out.data(), t, sizeof(double) * n, cudaMemcpyDeviceToHost, P->st));
    CK(cudaStreamSynchronize(P->st));
  } else {
    std::memcpy(out.data(), t, sizeof(double) * n);
  }
  for (double v : out)
    if (!std::isfinite(v)) throw CudaFail{OCTMC_ERR_INVALID_ARG};
  return out;
}

void create_impl(octmc_problem* P) {
  const octmc_desc& D = P->desc;
  check_device();
  const int L = D.levels;
  const int dt = D.storage;
  P->lv.resize(L);
  int w = D.w, h = D.h, d = D.d;
  std::vector<double> tx = fetch_times(P, D.tx, (size_t)w * h), ty = fetch_times(P, D.ty, (size_t)w * h);
  // The pyramid is built in float32; with 16-bit storage every level is
  // rounded once (to nearest even) from its float32 box means, and the
  // float32 copies are temporaries (kept in P->temps until released).
  float* prev32[2] = {nullptr, nullptr};
  for (int l = 0; l < L; l++) {
    LevelDev& X = P->lv[l].dev;
    X.w = w; X.h = h; X.d = d; X.dp = pad4(d);
    X.dtype = dt;
    const int64_t cols = (int64_t)w * h;
    float* cur32[2];
    for (int V = 0; V < 2; V++) {
      cur32[V] = dalloc<float>((size_t)cols * X.dp);
      if (dt != OCTMC_F32) P->temps.push_back(cur32[V]);
    }
    if (P->have_ang) {
      X.ax = dalloc<float>((size_t)cols);
      X.ay = dalloc<float>((size_t)cols);
    }
    if (D.vx) X.vx = dalloc<float>((size_t)h);
    if (D.vy) X.vy = dalloc<float>((size_t)w);
    if (l == 0) {
      upload_volume(P, D.sx, cur32[0], w, h, d, X.dp);
      upload_volume(P, D.sy, cur32[1], w, h, d, X.dp);
      if (P->have_ang) {
        upload(P, D.ax, X.ax, (size_t)cols);
        upload(P, D.ay, X.ay, (size_t)cols);
      }
      if (D.vx) upload(P, D.vx, X.vx, (size_t)h);
      if (D.vy) upload(P, D.vy, X.vy, (size_t)w);
    } else {
      const LevelDev& F = P->lv[l - 1].dev;
      for (int V = 0; V < 2; V++)
        CK(launch_pyr_volume(prev32[V], F.w, F.h, F.d, F.dp, cur32[V], w, h, d, X.dp, P->st));
      if (P->have_ang) {
        CK(launch_pyr_image(F.ax, F.w, F.h, X.ax, P->st));
        CK(launch_pyr_image(F.ay, F.w, F.h, X.ay, P->st));
      }
      if (X.vx) CK(launch_pyr_line(F.vx, F.h, X.vx, P->st));
      if (X.vy) CK(launch_pyr_line(F.vy, F.w, X.vy, P->st));
      tx = time_down(tx, F.w, F.h);
      ty = time_down(ty, F.w, F.h);
    }
    if (dt == OCTMC_F32) {
      X.sx = cur32[0];
      X.sy = cur32[1];
    } else {
      X.sx = dalloc<uint16_t>((size_t)cols * X.dp);
      X.sy = dalloc<uint16_t>((size_t)cols * X.dp);
      CK(launch_convert(cur32[0], X.sx, dt, cols * X.dp, P->st));
      CK(launch_convert(cur32[1], X.sy, dt, cols * X.dp, P->st));
    }
    prev32[0] = cur32[0];
    prev32[1] = cur32[1];
    for (int V = 0; V < 2; V++) {
      std::vector<int> pv, nx;
      std::vector<float> wp, wn;
      build_chain(V == 0 ? tx : ty, pv, nx, wp, wn);
      X.prev[V] = dalloc<int>((size_t)cols);
      X.next[V] = dalloc<int>((size_t)cols);
      X.wprev[V] = dalloc<float>((size_t)cols);
      X.wnext[V] = dalloc<float>((size_t)cols);
      upload_host(P, pv, X.prev[V]);
      upload_host(P, nx, X.next[V]);
      upload_host(P, wp, X.wprev[V]);
      upload_host(P, wn, X.wnext[V]);
      CK(cudaStreamSynchronize(P->st));  // host vectors go out of scope
    }
    P->lv[l].mu = D.mu > 0 ? D.mu : 1.0 / (2.0 * (double)w * (double)h);
    w = half_up(w);
    h = half_up(h);
    d = half_up(d);
  }
  const int64_t n0 = P->plane(0);
  P->str = dalloc<float>((size_t)n0);
  P->ang = dalloc<float>((size_t)n0);
  P->gdata = dalloc<float>((size_t)6 * n0);
  P->partials = dalloc<double>((size_t)8 * std::max(reg_grid_blocks(n0), msum_grid_blocks()));
  P->counters = dalloc<unsigned>(2);
  CK(cudaMemsetAsync(P->counters, 0, 2 * sizeof(unsigned), P->st));
  P->res = dalloc<EvalResult>(1);
  CK(cudaMallocHost(&P->res_host, sizeof(EvalResult)));
  CK(cudaStreamSynchronize(P->st));
  for (void* t : P->temps) dfree(t);
  P->temps.clear();
}

void collect_profile(octmc_problem* P) {
  if (!P->prof_pending) return;
  float ms = 0.f;
  CK(cudaEventSynchronize(P->ev1));
  CK(cudaEventElapsedTime(&ms, P->ev0, P->ev1));
  P->prof_ms += ms;
  P->prof_count++;
  P->prof_pending = false;
}

// ------------------------------------------------------------ evaluation
// One objective (+ gradient) evaluation request.
struct EvalReq {
  octmc_problem* P;
  int level;
  const double* x;
  double* grad;       // null: objective only
  const double* dir;  // null: no grad . dir
  double eta;
  double delta0;
  bool async = false;           // no host copy of the result (the caller does not wait)
  double* terms_dev = nullptr;  // if set: the 6 result terms copied here (device)
};

// A non-blocking side stream with its fork/join events, one per thread and
// device (created on first use, kept for the life of the thread).
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
SideStream& side_stream() {
  thread_local std::map<int, SideStream> per_device;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  SideStream& ss = per_device[dev];
  if (!ss.s) {
    CK(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming));
  }
  return ss;
}

// Enqueues the evaluations of several problems as one batch: msum, data
// (one launch per storage dtype) and reg kernels over all of them, then the
// copy of every EvalResult to its problem's pinned host copy.  A problem
// may appear once per batch.  Every request gets the same blocks, partition
// and reduction order as when it is evaluated alone, so its results do not
// depend on the batch.  The caller synchronises the stream.
void eval_batch(cudaStream_t st, const std::vector<EvalReq>& reqs) {
  for (size_t c0 = 0; c0 < reqs.size(); c0 += kMaxSlots) {
    const int ns = (int)std::min<size_t>(kMaxSlots, reqs.size() - c0);
    thread_local static MsumMulti MM;
    thread_local static RegMulti RM;
    thread_local static DataMulti DM[3];
    MM.nslots = RM.nslots = ns;
    MM.b0[0] = RM.b0[0] = 0;
    int nd[3] = {0, 0, 0};
    for (int k = 0; k < ns; k++) {
      const EvalReq& q = reqs[c0 + k];
      octmc_problem* P = q.P;
      const Level& Lv = P->lv[q.level];
      const int64_t n = (int64_t)Lv.dev.w * Lv.dev.h;
      MsumSlot& ms = MM.sl[k];
      ms.disp = q.x;
      ms.plane = n;
      ms.res = P->res;
      ms.partials = P->partials;
      ms.counter = P->counters + 0;
      MM.b0[k + 1] = MM.b0[k] + msum_grid_blocks();
      DataArgs A;
      A.L = Lv.dev;
      A.disp = q.x;
      A.str_out = P->str;
      A.ang_out = P->ang;
      A.grad = q.grad ? P->gdata : nullptr;
      A.eta = q.eta;
      A.eta_dev = nullptr;
      A.delta0 = P->have_ang ? q.delta0 : 0.0;
      A.eps_h = (float)P->desc.eps_h;
      A.loss = P->desc.loss;
      const int dt = Lv.dev.dtype;
      DM[dt].da[nd[dt]++] = A;
      RegArgs& R = RM.ra[k];
      R.L = Lv.dev;
      R.disp = q.x;
      R.grad = q.grad;
      R.gdata = P->gdata;
      R.dir = q.dir;
      R.str_in = P->str;
      R.ang_in = P->ang;
      R.alpha = P->desc.alpha;
      R.eps_r = P->desc.eps_r;
      R.mu = Lv.mu;
      R.eta = q.eta;
      R.eta_dev = nullptr;
      R.result = P->res;
      R.partials = P->partials;
      R.counter = P->counters + 1;
      R.ctl = nullptr;
      R.h_branch = 0;
      RM.b0[k + 1] = RM.b0[k] + reg_grid_blocks(n);
    }
    // The mean-term sums only feed the regulariser kernel: they run on a side
    // stream, overlapped with the data kernel, and are joined before it.
    SideStream& ss = side_stream();
    CK(cudaEventRecord(ss.fork, st));
    CK(cudaStreamWaitEvent(ss.s, ss.fork, 0));
    CK(launch_msum_multi(MM, ss.s));
    CK(cudaEventRecord(ss.join, ss.s));
    octmc_problem* P0 = reqs[c0].P;
    const bool prof = (ns == 1 && P0->profile && !reqs[c0].async);
    if (prof) CK(cudaEventRecord(P0->ev0, st));
    for (int dt = 0; dt < 3; dt++) {
      if (!nd[dt]) continue;
      DM[dt].nslots = nd[dt];
      CK(launch_data_multi(DM[dt], dt, st));
    }
    if (prof) {
      CK(cudaEventRecord(P0->ev1, st));
      P0->prof_pending = true;
    }
    CK(cudaStreamWaitEvent(st, ss.join, 0));
    CK(launch_reg_multi(RM, st));
    for (int k = 0; k < ns; k++) {
      const EvalReq& q = reqs[c0 + k];
      if (q.terms_dev)
        CK(cudaMemcpyAsync(q.terms_dev, q.P->res->terms, sizeof(double) * 6, cudaMemcpyDeviceToDevice, st));
      if (!q.async) CK(cudaMemcpyAsync(q.P->res_host, q.P->res, sizeof(EvalResult), cudaMemcpyDeviceToHost, st));
    }
  }
}

void collect_profiles(const std::vector<EvalReq>& reqs) {
  for (const EvalReq& q : reqs)
    if (q.P->profile) collect_profile(q.P);
}

// One evaluation of one problem, synchronised (results in P->res_host).
void eval_impl(octmc_problem* P, int l, const double* disp, double* grad, const double* dir, double eta,
               double delta0, bool sync) {
  std::vector<EvalReq> r{{P, l, disp, grad, dir, eta, delta0}};
  eval_batch(P->st, r);
  if (sync) {
    CK(cudaStreamSynchronize(P->st));
    collect_profiles(r);
  }
}

double eta_from(const EvalResult& r) {
  const double s = r.terms[0], a = r.terms[1];
  const double e = std::sqrt(a / s);
  if (!(s > 0) || !(a > 0) || !std::isfinite(e)) return 1.0;
  return e;
}

double eta_impl(octmc_problem* P, int l, const double* disp0) {
  if (!P->have_ang) return 1.0;
  eval_impl(P, l, disp0, nullptr, nullptr, 1.0, 0.5, true);
  return eta_from(*P->res_host);
}

void ensure_solver(octmc_problem* P) {
  if (P->x) return;
  const size_t n = (size_t)6 * P->plane(0);
  P->x = dalloc<double>(n);
  P->g = dalloc<double>(n);
  P->xt = dalloc<double>(n);
  P->gt = dalloc<double>(n);
  P->xb = dalloc<double>(n);
  P->gb = dalloc<double>(n);
  P->dir = dalloc<double>(n);
  P->opt = new octmc_lbfgs();
  P->opt->init((int64_t)n, P->desc.lbfgs_m, P->st);
}

// ------------------------------------------------------------ device-resident solve
// A solve is one CUDA graph.  Per level: the start-field evaluation for eta
// (Eq. 10), a one-thread kernel that sets eta and the controller state, and
// a WHILE node whose body evaluates one trial point (trial kernel, which
// also saves the previous trial when the line search kept it as its best
// point; mean-term sums forked onto a side stream, data kernel, regulariser
// kernel with the line-search decision in its last block) and, under an IF
// node set by that decision, the accepted-step branch (history pair from the
// trial or the restored best point, products and compact-form direction,
// direction); a stats
// kernel closes the level, and the next finer level starts with the
// prolongation.  The host launches the graph once, synchronises once and
// reads the per-level statistics.  Graphs are built on first use and kept
// with the problem (their kernels' arguments do not change between solves).
void ensure_device_solver(octmc_problem* P) {
  ensure_solver(P);
  if (P->sstate) return;
  const int m = P->desc.lbfgs_m;
  P->sstate = dalloc<SolveState>(1);
  P->lstats = dalloc<LevelStatsDev>(16);
  CK(cudaMallocHost(&P->lstats_host, 16 * sizeof(LevelStatsDev)));
  const int64_t n0 = 6 * P->plane(0);
  const size_t nout = (size_t)(2 * (2 * m + 2) + 3);
  P->spartials = dalloc<double>(nout * (size_t)solve_dots_blocks(n0));
  P->scounter = dalloc<unsigned>(1);
  CK(cudaMemsetAsync(P->scounter, 0, sizeof(unsigned), P->st));
  if (P->desc.persistent_ascans > 0 && P->plane(P->lv.size() - 1) <= P->desc.persistent_ascans) {
    P->lgrid = level_grid(P->desc.storage);
    if (P->lgrid > 0) {
      P->lpart = dalloc<double>((size_t)level_part_doubles(P->lgrid));
      P->lbar = dalloc<unsigned>(4);
    }
  }
  CK(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&P->cap_side, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&P->cap_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->cap_join, cudaEventDisableTiming));
  CK(cudaStreamSynchronize(P->st));
}

// Captures launch(stream) into graph g after the node `dep` (none if null)
// and returns the capture's single leaf node.
template <typename F>
cudaGraphNode_t capture_after(octmc_problem* P, cudaGraph_t g, cudaGraphNode_t dep, F&& launch) {
  cudaStream_t cs = P->cap;
  CK(cudaStreamBeginCaptureToGraph(cs, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, cudaStreamCaptureModeRelaxed));
  launch(cs);
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  if (ndeps != 1) throw CudaFail{OCTMC_ERR_CUDA};
  const cudaGraphNode_t leaf = deps[0];
  cudaGraph_t out = g;
  CK(cudaStreamEndCapture(cs, &out));
  return leaf;
}

// msum (side stream) + data + reg at the level's current x or trial point
// With ctl (inside a level's loop) the mean-term sums are not launched here:
// the trial kernel forms them with the trial point.
void capture_eval(octmc_problem* P, cudaStream_t cs, int l, const double* x, double* grad, const double* dir,
                  double eta, const double* eta_dev, double delta0, SolveState* ctl,
                  cudaGraphConditionalHandle hb, cudaGraphConditionalHandle hw) {
  const Level& Lv = P->lv[l];
  const int64_t plane = P->plane(l);
  if (!ctl) {
    CK(cudaEventRecord(P->cap_fork, cs));
    CK(cudaStreamWaitEvent(P->cap_side, P->cap_fork, 0));
    CK(launch_msum(x, plane, P->res, P->partials, P->counters + 0, P->cap_side));
    CK(cudaEventRecord(P->cap_join, P->cap_side));
  }
  DataArgs A;
  std::memset(&A, 0, sizeof(A));
  A.L = Lv.dev;
  A.disp = x;
  A.str_out = P->str;
  A.ang_out = P->ang;
  A.grad = grad ? P->gdata : nullptr;
  A.eta = eta;
  A.eta_dev = eta_dev;
  A.delta0 = P->have_ang ? delta0 : 0.0;
  A.eps_h = (float)P->desc.eps_h;
  A.loss = P->desc.loss;
  CK(launch_data(A, cs));
  if (!ctl) CK(cudaStreamWaitEvent(cs, P->cap_join, 0));
  RegArgs R;
  std::memset(&R, 0, sizeof(R));
  R.L = Lv.dev;
  R.disp = x;
  R.grad = grad;
  R.gdata = P->gdata;
  R.dir = dir;
  R.str_in = P->str;
  R.ang_in = P->ang;
  R.alpha = P->desc.alpha;
  R.eps_r = P->desc.eps_r;
  R.mu = Lv.mu;
  R.eta = eta;
  R.eta_dev = eta_dev;
  R.result = P->res;
  R.partials = P->partials;
  R.counter = P->counters + 1;
  R.ctl = ctl;
  R.h_branch = hb;
  R.h_while = hw;
  CK(launch_reg(R, cs));
}

// Appends the nodes of one level solve (x holds the start field) after
// `dep`; returns the level's last node.
cudaGraphNode_t append_level(octmc_problem* P, cudaGraph_t g, cudaGraphNode_t dep, int l, int stats_slot) {
  const int64_t n = 6 * P->plane(l);
  const int m = P->desc.lbfgs_m;
  const octmc_desc& D = P->desc;
  SolveState* S = P->sstate;
  HistSet H{};
  for (int b = 0; b <= m; b++) {
    H.S[b] = P->opt->S[b];
    H.Y[b] = P->opt->Y[b];
  }
  SolveCfg cfg{};
  cfg.n = n;
  cfg.m = m;
  cfg.max_iter = D.max_iter;
  cfg.max_ls = D.max_ls;
  cfg.max_evals = (int)std::min<int64_t>((int64_t)D.max_iter * (D.max_ls + 1) + 8, 1 << 30);
  cfg.gtol = D.gtol;
  cfg.ftol = D.ftol;
  cfg.have_ang = P->have_ang ? 1 : 0;
  // start-field evaluation for eta, the level's state, a zero direction
  dep = capture_after(P, g, dep, [&](cudaStream_t cs) {
    if (P->have_ang) capture_eval(P, cs, l, P->x, nullptr, nullptr, 1.0, nullptr, 0.5, nullptr, 0, 0);
    CK(launch_solve_level_init(S, P->res, cfg, cs));
    CK(cudaMemsetAsync(P->dir, 0, sizeof(double) * n, cs));
  });
  SolveVecs V{P->x, P->g, P->xt, P->gt, P->xb, P->gb, P->dir, n, P->plane(l)};
  if (P->lgrid > 0 && P->plane(l) <= P->desc.persistent_ascans) {
    // a small level: its whole loop in one cooperative kernel
    const Level& Lv = P->lv[l];
    LevelArgs LA;
    std::memset(&LA, 0, sizeof(LA));
    LA.S = S;
    LA.H = H;
    LA.V = V;
    LA.D.L = Lv.dev;
    LA.D.disp = P->xt;
    LA.D.str_out = P->str;
    LA.D.ang_out = P->ang;
    LA.D.grad = P->gdata;
    LA.D.eta = 1.0;
    LA.D.eta_dev = &S->eta;
    LA.D.delta0 = P->have_ang ? D.delta0 : 0.0;
    LA.D.eps_h = (float)D.eps_h;
    LA.D.loss = D.loss;
    LA.alpha = D.alpha;
    LA.eps_r = D.eps_r;
    LA.mu = Lv.mu;
    LA.part = P->lpart;
    LA.bar = P->lbar;
    LA.err = reinterpret_cast<int*>(P->lbar + 2);
    return capture_after(P, g, dep, [&](cudaStream_t cs) {
      CK(cudaMemsetAsync(P->lbar, 0, 4 * sizeof(unsigned), cs));
      CK(launch_level_persistent(LA, Lv.dev.dtype, cs));
      CK(launch_solve_level_stats(S, P->lstats + stats_slot, cs));
    });
  }
  // the iteration loop
  cudaGraphConditionalHandle hw, hb;
  CK(cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  CK(cudaGraphAddNode(&wnode, g, &dep, nullptr, 1, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  CK(cudaGraphConditionalHandleCreate(&hb, body, 0, cudaGraphCondAssignDefault));
  const double* eta_dev = &S->eta;
  const cudaGraphNode_t sink = capture_after(P, body, nullptr, [&](cudaStream_t cs) {
    CK(launch_solve_trial(S, H, V, P->res, P->partials, P->counters + 0, cs));
    capture_eval(P, cs, l, P->xt, P->gt, P->dir, 1.0, eta_dev, D.delta0, S, hb, hw);
  });
  cudaGraphNodeParams ip{};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hb;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t inode;
  CK(cudaGraphAddNode(&inode, body, &sink, nullptr, 1, &ip));
  capture_after(P, ip.conditional.phGraph_out[0], nullptr, [&](cudaStream_t cs) {
    CK(launch_solve_dots(S, H, m, V, P->spartials, P->scounter, cs));
  });
  // the level's last iterate, and its statistics
  return capture_after(P, g, wnode, [&](cudaStream_t cs) {
    CK(launch_solve_finish(S, V, cs));
    CK(launch_solve_level_stats(S, P->lstats + stats_slot, cs));
  });
}

// The graph solving levels `first` down to `last` (x holds the start field
// of `first`; each finer level starts from the prolonged result).
cudaGraphExec_t solve_graph(octmc_problem* P, int first, int last) {
  const int key = first * 64 + last;
  auto it = P->graphs.find(key);
  if (it != P->graphs.end()) return it->second.second;
  ensure_device_solver(P);
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphExec_t ex = nullptr;
  try {
    cudaGraphNode_t dep = nullptr;
    for (int l = first; l >= last; l--) {
      if (l != first) {
        const LevelDev& C = P->lv[l + 1].dev;
        const LevelDev& F = P->lv[l].dev;
        const int64_t nf = 6 * P->plane(l);
        dep = capture_after(P, g, dep, [&](cudaStream_t cs) {
          CK(launch_prolong(P->x, C.w, C.h, P->xt, F.w, F.h, cs));
          CK(cudaMemcpyAsync(P->x, P->xt, sizeof(double) * nf, cudaMemcpyDeviceToDevice, cs));
        });
      }
      dep = append_level(P, g, dep, l, first - l);
    }
    CK(cudaGraphInstantiate(&ex, g, 0));
  } catch (...) {
    cudaStreamCaptureStatus cst;
    if (cudaStreamIsCapturing(P->cap, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(P->cap, &junk);
      if (junk && junk != g) cudaGraphDestroy(junk);
    }
    cudaGraphDestroy(g);
    cudaGetLastError();
    throw;
  }
  P->graphs[key] = {g, ex};
  return ex;
}

// Enqueues a solve of levels first..last on P's stream: x from `init`
// (level `first` layout; null: zero), the result copied to `out`.
void launch_solve(octmc_problem* P, int first, int last, const double* init, double* out) {
  cudaGraphExec_t ex = solve_graph(P, first, last);
  const int64_t n = 6 * P->plane(first);
  if (init) CK(cudaMemcpyAsync(P->x, init, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->st));
  else CK(cudaMemsetAsync(P->x, 0, sizeof(double) * n, P->st));
  CK(cudaGraphLaunch(ex, P->st));
  const int nl = first - last + 1;
  CK(cudaMemcpyAsync(P->lstats_host, P->lstats, nl * sizeof(LevelStatsDev), cudaMemcpyDeviceToHost, P->st));
  if (out) CK(cudaMemcpyAsync(out, P->x, sizeof(double) * 6 * P->plane(last), cudaMemcpyDeviceToDevice, P->st));
}

// Statistics and return code of a finished launch_solve (stream synchronised).
int finish_solve(octmc_problem* P, int first, int last, octmc_stats* st) {
  int rc = OCTMC_OK;
  for (int k = 0; k < first - last + 1; k++) {
    const LevelStatsDev& L = P->lstats_host[k];
    if (st) {
      st[k] = octmc_stats{};
      st[k].level = first - k;
      st[k].iters = L.iters;
      st[k].evals = L.evals;
      st[k].status = L.status;
      st[k].f = L.f;
      st[k].eta = L.eta;
      st[k].seconds = (double)(L.t_end - L.t_start) * 1e-9;
    }
    P->lv[first - k].eta = L.eta;
    if (L.status == 3) rc = OCTMC_ERR_TIMEOUT;
    else if (!std::isfinite(L.f) && rc != OCTMC_ERR_TIMEOUT) rc = OCTMC_ERR_NONFINITE;
    else if (L.status == 1 && rc == OCTMC_OK) rc = OCTMC_NOT_CONVERGED;
  }
  return rc;
}

int solve_impl(octmc_problem* P, int l, double* disp_inout, octmc_stats* st) {
  launch_solve(P, l, l, disp_inout, disp_inout);
  CK(cudaStreamSynchronize(P->st));
  return finish_solve(P, l, l, st);
}

// ------------------------------------------------------------ prealignment
// Stage 1 of Sec. 2.1: L-BFGS over the per-B-scan axial offsets and tilts
// (2 (w + h) values per level), with the same line search and stopping rules
// as the 3-D solve; each evaluation maps the parameters to the field, runs
// the objective with the structural term alone (delta_0 = 0, eta = 1) and
// reduces the field gradient to the parameters.
int prealign_n(const octmc_problem* P, int l) { return 2 * (P->lv[l].dev.w + P->lv[l].dev.h); }

void ensure_prealign(octmc_problem* P) {
  ensure_solver(P);
  if (P->pre_D) return;
  const size_t n = (size_t)6 * P->plane(0);
  P->pre_D = dalloc<double>(n);
  P->pre_G = dalloc<double>(n);
  P->pre_aux = dalloc<double>(2);
  P->pre_prm = dalloc<double>((size_t)prealign_n(P, 0));
  CK(cudaMallocHost(&P->pre_aux_host, 2 * sizeof(double)));
}

// f (host) and, if gprm, the parameter gradient (device); with dir also
// gprm . dir in *gdir.
void prealign_eval_impl(octmc_problem* P, int l, const double* prm, double* gprm, const double* dir, double* f,
                        double* gdir) {
  ensure_prealign(P);
  const LevelDev& L = P->lv[l].dev;
  CK(launch_prm_to_disp(prm, L.w, L.h, P->pre_D, P->st));
  eval_batch(P->st, {EvalReq{P, l, P->pre_D, gprm ? P->pre_G : nullptr, nullptr, 1.0, 0.0}});
  if (gprm) {
    CK(launch_grad_to_prm(P->pre_G, L.w, L.h, prm, gprm, P->pre_aux, P->st));
    if (dir) CK(launch_prm_dot(gprm, dir, prealign_n(P, l), P->pre_aux + 1, P->st));
  } else {
    // T alone: reduce a zero field gradient into scratch
    CK(cudaMemsetAsync(P->pre_G, 0, sizeof(double) * 6 * P->plane(l), P->st));
    CK(launch_grad_to_prm(P->pre_G, L.w, L.h, prm, P->pre_prm, P->pre_aux, P->st));
  }
  CK(cudaMemcpyAsync(P->pre_aux_host, P->pre_aux, 2 * sizeof(double), cudaMemcpyDeviceToHost, P->st));
  CK(cudaStreamSynchronize(P->st));
  *f = P->res_host->terms[4] + P->pre_aux_host[0];
  if (gdir) *gdir = P->pre_aux_host[1];
}

int prealign_level_impl(octmc_problem* P, int l, double* prm, octmc_stats* st) {
  ensure_prealign(P);
  const auto t0 = std::chrono::steady_clock::now();
  const octmc_desc& D = P->desc;
  const int n = prealign_n(P, l);
  octmc_lbfgs* O = P->opt;
  O->n = n;
  O->reset();
  double *x = P->x, *g = P->g, *xt = P->xt, *gt = P->gt, *xb = P->xb, *gb = P->gb, *dir = P->dir;
  CK(cudaMemcpyAsync(x, prm, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->st));
  double f;
  prealign_eval_impl(P, l, x, g, nullptr, &f, nullptr);
  int evals = 1, iters = 0, status = 1, small = 0, retried = 0;
  O->prepare(g, false);
  while (iters < D.max_iter) {
    if (O->gmax <= D.gtol) {
      status = 0;
      break;
    }
    const double dg0 = O->direction(g, dir);
    double a = (O->k() == 0) ? 1.0 / std::sqrt(O->gg) : 1.0;
    double lo = 0.0, hi = std::numeric_limits<double>::infinity(), ft = 0.0, fb = 0.0;
    bool accepted = false, have_lo = false;
    for (int ls = 0; ls < D.max_ls; ls++) {
      CK(launch_axpy(x, a, dir, xt, n, P->st));
      double dgt;
      prealign_eval_impl(P, l, xt, gt, dir, &ft, &dgt);
      evals++;
      if (!(ft <= f + 1e-4 * a * dg0)) {
        hi = a;
        a = 0.5 * (lo + hi);
      } else if (dgt < 0.9 * dg0) {
        lo = a;
        have_lo = true;
        fb = ft;
        std::swap(xb, xt);
        std::swap(gb, gt);
        a = std::isinf(hi) ? 2.0 * a : 0.5 * (lo + hi);
      } else {
        accepted = true;
        break;
      }
    }
    if (!accepted) {
      if (have_lo) {
        std::swap(xt, xb);
        std::swap(gt, gb);
        ft = fb;
      } else if (O->k() > 0 && !retried) {
        O->reset();
        retried = 1;
        O->prepare(g, false);
        continue;
      } else {
        status = 2;
        break;
      }
    }
    retried = 0;
    CK(launch_sub2(xt, x, gt, g, O->S[O->spare], O->Y[O->spare], n, P->st));
    const double rel = (f - ft) / std::max(std::max(std::fabs(f), std::fabs(ft)), 1.0);
    std::swap(x, xt);
    std::swap(g, gt);
    f = ft;
    iters++;
    small = (rel < D.ftol) ? small + 1 : 0;
    O->prepare(g, true);
    if (small >= 3) {
      status = 0;
      break;
    }
  }
  CK(cudaMemcpyAsync(prm, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->st));
  CK(cudaStreamSynchronize(P->st));
  if (st) {
    *st = octmc_stats{};
    st->level = l;
    st->iters = iters;
    st->evals = evals;
    st->status = status;
    st->f = f;
    st->eta = 1.0;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!std::isfinite(f)) return OCTMC_ERR_NONFINITE;
  return status == 1 ? OCTMC_NOT_CONVERGED : OCTMC_OK;
}

template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const CudaFail& e) {
    cudaGetLastError();
    return e.code;
  } catch (const std::bad_alloc&) {
    return OCTMC_ERR_OOM;
  } catch (...) {
    return OCTMC_ERR_CUDA;
  }
}

bool valid_level(const octmc_problem* p, int level) { return p && level >= 0 && level < (int)p->lv.size(); }

}  // namespace

// ====================================================================== server
// Continuous batching of independent solves: requests wait in a FIFO queue
// and are admitted (their problem created on the device, their whole solve
// launched as one device-resident graph on a stream of their own) while a
// slot is free and their estimated device memory fits the budget.  The
// graphs of all admitted requests run concurrently; the GPU interleaves
// their kernels, and a request that arrives while others run starts at
// once.  A request's kernels and reductions are those of a solve of it
// alone, so its result does not depend on the mix.  Each step admits what
// fits and retires finished requests without blocking; finished results
// stay on the device until polled.
namespace {

int64_t estimate_bytes_impl(const octmc_desc& D) {
  int64_t w = D.w, h = D.h, d = D.d, total = 0, peak_tmp = 0;
  const int64_t sbytes = D.storage == OCTMC_F32 ? 4 : 2;
  const int64_t n0 = w * h;
  for (int l = 0; l < std::max(D.levels, 1); l++) {
    const int64_t cols = w * h, dp = (d + 3) & ~int64_t(3);
    total += 2 * cols * dp * sbytes + cols * (2 * 4 + 2 * (4 + 4 + 4 + 4)) + (w + h) * 4;
    if (D.storage != OCTMC_F32) peak_tmp += 2 * cols * dp * 4;
    w = (w + 1) / 2;
    h = (h + 1) / 2;
    d = (d + 1) / 2;
  }
  const int64_t m = std::max(D.lbfgs_m, 1);
  total += n0 * (4 + 4 + 24);                                // per-A-scan partials, float gradient
  total += (7 + 1) * 6 * n0 * 8 + 2 * (m + 1) * 6 * n0 * 8;  // solver vectors, result, history
  total += 1 << 20;                                          // small buffers, solver state
  return total + peak_tmp;
}

}  // namespace

struct octmc_server {
  struct Req {
    int64_t ticket;
    octmc_desc desc;
    int64_t bytes;
    octmc_problem* P = nullptr;
    double* result = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<octmc_stats> stats;
    int state = OCTMC_REQ_QUEUED;
    int rc = OCTMC_OK;
  };
  cudaStream_t st = nullptr;  // the caller's stream: results are copied out on it
  int64_t budget = 0, in_use = 0;
  int max_slots = 1;
  int64_t next_ticket = 1;
  std::deque<std::shared_ptr<Req>> queue;
  std::vector<std::shared_ptr<Req>> active;
  std::map<int64_t, std::shared_ptr<Req>> all;
  // released requests whose device memory is freed once nothing runs:
  // freeing synchronises the device, which would stall the running solves
  std::vector<std::shared_ptr<Req>> graveyard;

  static void free_now(Req& r) {
    if (r.stream) cudaStreamSynchronize(r.stream);
    delete r.P;
    r.P = nullptr;
    dfree(r.result);
    r.result = nullptr;
    if (r.done) cudaEventDestroy(r.done);
    r.done = nullptr;
    if (r.stream) cudaStreamDestroy(r.stream);
    r.stream = nullptr;
  }

  void release(const std::shared_ptr<Req>& r) {
    if (active.empty()) {
      free_now(*r);
      in_use -= r->bytes;
      r->bytes = 0;
    } else {
      graveyard.push_back(r);
    }
  }

  void bury() {
    if (!active.empty()) return;
    for (auto& r : graveyard) {
      free_now(*r);
      in_use -= r->bytes;
      r->bytes = 0;
    }
    graveyard.clear();
  }

  ~octmc_server() {
    for (auto& r : active)
      if (r->stream) cudaStreamSynchronize(r->stream);
    active.clear();
    for (auto& kv : all) free_now(*kv.second);
    for (auto& r : graveyard) free_now(*r);
  }

  void admit() {
    while (!queue.empty() && (int)active.size() < max_slots) {
      auto r = queue.front();
      if (in_use + r->bytes > budget) break;  // wait for memory (finished results count until polled)
      queue.pop_front();
      in_use += r->bytes;
      try {
        CK(cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming));
        octmc_desc D = r->desc;
        D.stream = r->stream;
        r->P = new octmc_problem();
        r->P->desc = D;
        r->P->st = r->stream;
        r->P->have_ang = (D.ax != nullptr);
        create_impl(r->P);
        r->result = dalloc<double>((size_t)6 * D.w * D.h);
        launch_solve(r->P, D.levels - 1, 0, nullptr, r->result);
        CK(cudaEventRecord(r->done, r->stream));
        r->state = OCTMC_REQ_RUNNING;
        active.push_back(r);
      } catch (const CudaFail& e) {
        cudaGetLastError();
        r->rc = e.code;
        r->state = OCTMC_REQ_DONE;
        release(r);
      }
    }
  }

  void step() {
    std::vector<std::shared_ptr<Req>> still;
    for (auto& r : active) {
      const cudaError_t q = cudaEventQuery(r->done);
      if (q == cudaErrorNotReady) {
        still.push_back(r);
        continue;
      }
      if (q != cudaSuccess) {
        cudaGetLastError();
        r->rc = OCTMC_ERR_CUDA;
      } else {
        const int L = r->desc.levels;
        r->stats.assign(L, octmc_stats{});
        r->rc = finish_solve(r->P, L - 1, 0, r->stats.data());
      }
      r->state = OCTMC_REQ_DONE;
    }
    active.swap(still);
    bury();
    admit();
  }
};

// ====================================================================== C ABI
extern "C" {

void octmc_desc_defaults(octmc_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->storage = OCTMC_F32;
  d->alpha = 0.1;
  d->delta0 = 0.5;
  d->eps_h = 1e-3;
  d->eps_r = 1e-2;
  d->mu = 0.0;
  d->loss = OCTMC_LOSS_PSEUDO_HUBER;
  d->levels = 1;
  d->lbfgs_m = 8;
  d->max_iter = 5000;
  d->max_ls = 20;
  d->gtol = 1e-6;
  d->ftol = 1e-7;
  d->persistent_ascans = 0;
}

int octmc_create_problem(const octmc_desc* desc, octmc_problem** out) {
  if (!desc || !out) return OCTMC_ERR_INVALID_ARG;
  *out = nullptr;
  const octmc_desc& D = *desc;
  if (D.w < 1 || D.h < 1 || D.d < 1 || !D.sx || !D.sy || !D.tx || !D.ty) return OCTMC_ERR_INVALID_ARG;
  if ((D.ax == nullptr) != (D.ay == nullptr)) return OCTMC_ERR_INVALID_ARG;
  if (D.levels < 1 || D.levels > 16 || D.lbfgs_m < 1 || D.lbfgs_m > 32 || D.max_ls < 1 || D.max_iter < 0 ||
      D.persistent_ascans < 0)
    return OCTMC_ERR_INVALID_ARG;
  if (D.loss != OCTMC_LOSS_PSEUDO_HUBER && D.loss != OCTMC_LOSS_SSD) return OCTMC_ERR_INVALID_ARG;
  if (!(D.eps_h > 0) || !(D.eps_r > 0) || !(D.alpha >= 0) || !(D.delta0 >= 0)) return OCTMC_ERR_INVALID_ARG;
  if ((int64_t)D.w * D.h * pad4(D.d) / 4 >= (int64_t)1 << 32) return OCTMC_ERR_INVALID_ARG;
  if (D.storage != OCTMC_F32 && D.storage != OCTMC_BF16 && D.storage != OCTMC_F16) return OCTMC_ERR_INVALID_ARG;
  octmc_problem* P = new (std::nothrow) octmc_problem();
  if (!P) return OCTMC_ERR_OOM;
  P->desc = D;
  P->st = (cudaStream_t)D.stream;
  P->have_ang = (D.ax != nullptr);
  const int rc = guarded([&] {
    create_impl(P);
    return OCTMC_OK;
  });
  if (rc != OCTMC_OK) {
    delete P;
    return rc;
  }
  *out = P;
  return OCTMC_OK;
}

void octmc_destroy_problem(octmc_problem* p) {
  if (!p) return;
  if (p->st) cudaStreamSynchronize(p->st);
  else cudaDeviceSynchronize();
  delete p;
}

int octmc_level_shape(const octmc_problem* p, int level, int* w, int* h, int* d) {
  if (!valid_level(p, level)) return OCTMC_ERR_INVALID_ARG;
  const LevelDev& L = p->lv[level].dev;
  if (w) *w = L.w;
  if (h) *h = L.h;
  if (d) *d = L.d;
  return OCTMC_OK;
}

int octmc_set_eta(octmc_problem* p, int level, double eta) {
  if (!valid_level(p, level) || !(eta > 0) || !std::isfinite(eta)) return OCTMC_ERR_INVALID_ARG;
  p->lv[level].eta = eta;
  return OCTMC_OK;
}

int octmc_compute_eta(octmc_problem* p, int level, const double* disp0, double* eta_out) {
  if (!valid_level(p, level) || !disp0) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    const double e = eta_impl(p, level, disp0);
    p->lv[level].eta = e;
    if (eta_out) *eta_out = e;
    return OCTMC_OK;
  });
}

int octmc_eval_terms(octmc_problem* p, int level, const double* disp, double* terms, double* grad) {
  if (!valid_level(p, level) || !disp) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    eval_impl(p, level, disp, grad, nullptr, p->lv[level].eta, p->desc.delta0, true);
    if (terms) std::memcpy(terms, p->res_host->terms, sizeof(double) * 6);
    return std::isfinite(p->res_host->terms[4]) ? OCTMC_OK : OCTMC_ERR_NONFINITE;
  });
}

int octmc_eval_objective_grad(octmc_problem* p, int level, const double* disp, double* f, double* grad) {
  double terms[6];
  const int rc = octmc_eval_terms(p, level, disp, terms, grad);
  if (f && (rc == OCTMC_OK || rc == OCTMC_ERR_NONFINITE)) *f = terms[4];
  return rc;
}

int octmc_eval_objective_grad_async(octmc_problem* p, int level, const double* disp, double* grad,
                                    double* terms_dev, void* stream) {
  if (!valid_level(p, level) || !disp) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    const cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : p->st;
    EvalReq q{p, level, disp, grad, nullptr, p->lv[level].eta, p->desc.delta0};
    q.async = true;
    q.terms_dev = terms_dev;
    eval_batch(st, std::vector<EvalReq>{q});
    CK(cudaGetLastError());
    return OCTMC_OK;
  });
}

int octmc_eval_batch(octmc_problem* const* problems, int count, const int* levels, const double* const* disp,
                     double* const* grad, double* f_host) {
  if (!problems || !levels || !disp || count < 1 || count > 4096) return OCTMC_ERR_INVALID_ARG;
  std::vector<EvalReq> reqs;
  reqs.reserve(count);
  for (int k = 0; k < count; k++) {
    octmc_problem* P = problems[k];
    if (!valid_level(P, levels[k]) || !disp[k]) return OCTMC_ERR_INVALID_ARG;
    for (int j = 0; j < k; j++)
      if (problems[j] == P) return OCTMC_ERR_INVALID_ARG;
    reqs.push_back({P, levels[k], disp[k], grad ? grad[k] : nullptr, nullptr, P->lv[levels[k]].eta,
                    P->desc.delta0});
  }
  return guarded([&] {
    for (int k = 0; k < count; k++) CK(cudaStreamSynchronize(problems[k]->st));
    cudaStream_t st = problems[0]->st;
    eval_batch(st, reqs);
    CK(cudaStreamSynchronize(st));
    bool finite = true;
    for (int k = 0; k < count; k++) {
      const double f = problems[k]->res_host->terms[4];
      if (f_host) f_host[k] = f;
      finite = finite && std::isfinite(f);
    }
    return finite ? OCTMC_OK : OCTMC_ERR_NONFINITE;
  });
}

int octmc_solve_level(octmc_problem* p, int level, double* disp, octmc_stats* st) {
  if (!valid_level(p, level) || !disp) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] { return solve_impl(p, level, disp, st); });
}

int octmc_prolong(octmc_problem* p, int level, const double* coarse, double* fine) {
  if (!valid_level(p, level) || level < 1 || !coarse || !fine) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    const LevelDev& C = p->lv[level].dev;
    const LevelDev& F = p->lv[level - 1].dev;
    CK(launch_prolong(coarse, C.w, C.h, fine, F.w, F.h, p->st));
    CK(cudaStreamSynchronize(p->st));
    return OCTMC_OK;
  });
}

int octmc_solve_full(octmc_problem* p, double* disp_out, octmc_stats* st) {
  if (!p || !disp_out) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    const int L = (int)p->lv.size();
    launch_solve(p, L - 1, 0, nullptr, disp_out);
    CK(cudaStreamSynchronize(p->st));
    return finish_solve(p, L - 1, 0, st);
  });
}

int octmc_merge(octmc_problem* p, const double* disp0, double beta, double tau, float* merged, float* cx,
                float* cy, float* weights, float* angio) {
  if (!valid_level(p, 0) || !disp0 || !(beta >= 0) || !std::isfinite(beta) || !(tau >= 0) || !(tau <= 1))
    return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    const LevelDev& L = p->lv[0].dev;
    float* wts = weights;
    if (merged || weights || angio) {
      if (!p->mcounts) p->mcounts = dalloc<unsigned long long>(2 * (size_t)p->plane(0));
      if (!wts && merged) wts = p->gdata;  // scratch of 6 w h floats, unused outside evaluations
      CK(launch_merge_weights(L, disp0, beta, tau, p->mcounts, wts, angio, p->st));
    }
    if (merged || cx || cy) CK(launch_resample_merge(L, disp0, wts, merged, cx, cy, p->st));
    CK(cudaStreamSynchronize(p->st));
    return OCTMC_OK;
  });
}

int octmc_prealign_disp(octmc_problem* p, int level, const double* prm, double* disp) {
  if (!valid_level(p, level) || !prm || !disp) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    const LevelDev& L = p->lv[level].dev;
    CK(launch_prm_to_disp(prm, L.w, L.h, disp, p->st));
    CK(cudaStreamSynchronize(p->st));
    return OCTMC_OK;
  });
}

int octmc_prealign_eval(octmc_problem* p, int level, const double* prm, double* f_host, double* grad_prm) {
  if (!valid_level(p, level) || !prm) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    double f;
    prealign_eval_impl(p, level, prm, grad_prm, nullptr, &f, nullptr);
    if (f_host) *f_host = f;
    return std::isfinite(f) ? OCTMC_OK : OCTMC_ERR_NONFINITE;
  });
}

int octmc_prealign_level(octmc_problem* p, int level, double* prm_inout, octmc_stats* st) {
  if (!valid_level(p, level) || !prm_inout) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] { return prealign_level_impl(p, level, prm_inout, st); });
}

int octmc_prealign_full(octmc_problem* p, double* prm_out, double* disp0_out, octmc_stats* st) {
  if (!p || !prm_out) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    ensure_prealign(p);
    const int L = (int)p->lv.size();
    // the parameters of the current level live in the caller's buffer
    // (level-0 sized); the coarse copy for the prolongation in pre_prm
    double* cur = prm_out;
    CK(cudaMemsetAsync(cur, 0, sizeof(double) * prealign_n(p, L - 1), p->st));
    int rc = OCTMC_OK;
    for (int l = L - 1; l >= 0; l--) {
      if (l != L - 1) {
        const LevelDev& C = p->lv[l + 1].dev;
        const LevelDev& F = p->lv[l].dev;
        double* tmp = p->pre_prm;
        CK(cudaMemcpyAsync(tmp, cur, sizeof(double) * prealign_n(p, l + 1), cudaMemcpyDeviceToDevice, p->st));
        CK(launch_prm_prolong(tmp, C.w, C.h, cur, F.w, F.h, p->st));
      }
      octmc_stats s{};
      const int r = prealign_level_impl(p, l, cur, &s);
      if (st) st[L - 1 - l] = s;
      if (r < 0) return r;
      if (r == OCTMC_NOT_CONVERGED) rc = r;
    }
    if (disp0_out) {
      const LevelDev& F = p->lv[0].dev;
      CK(launch_prm_to_disp(cur, F.w, F.h, disp0_out, p->st));
      CK(cudaStreamSynchronize(p->st));
    }
    return rc;
  });
}

int octmc_level_data(const octmc_problem* p, int level, float* sx, float* sy, float* ax, float* ay, float* vx,
                     float* vy) {
  if (!valid_level(p, level)) return OCTMC_ERR_INVALID_ARG;
  octmc_problem* q = const_cast<octmc_problem*>(p);
  return guarded([&] {
    const LevelDev& L = q->lv[level].dev;
    const int64_t cols = (int64_t)L.w * L.h;
    if (sx) CK(launch_unpad_depth(L.sx, L.dtype, cols, L.d, L.dp, sx, q->st));
    if (sy) CK(launch_unpad_depth(L.sy, L.dtype, cols, L.d, L.dp, sy, q->st));
    if (ax && L.ax) CK(cudaMemcpyAsync(ax, L.ax, sizeof(float) * cols, cudaMemcpyDeviceToDevice, q->st));
    if (ay && L.ay) CK(cudaMemcpyAsync(ay, L.ay, sizeof(float) * cols, cudaMemcpyDeviceToDevice, q->st));
    if (vx && L.vx) CK(cudaMemcpyAsync(vx, L.vx, sizeof(float) * L.h, cudaMemcpyDeviceToDevice, q->st));
    if (vy && L.vy) CK(cudaMemcpyAsync(vy, L.vy, sizeof(float) * L.w, cudaMemcpyDeviceToDevice, q->st));
    CK(cudaStreamSynchronize(q->st));
    return OCTMC_OK;
  });
}

int octmc_lbfgs_create(int64_t n, int m, void* stream, octmc_lbfgs** out) {
  if (!out || n < 1 || m < 1 || m > 32) return OCTMC_ERR_INVALID_ARG;
  *out = nullptr;
  octmc_lbfgs* h = new (std::nothrow) octmc_lbfgs();
  if (!h) return OCTMC_ERR_OOM;
  const int rc = guarded([&] {
    h->init(n, m, (cudaStream_t)stream);
    CK(cudaStreamSynchronize(h->st));
    return OCTMC_OK;
  });
  if (rc != OCTMC_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return OCTMC_OK;
}

void octmc_lbfgs_destroy(octmc_lbfgs* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  delete h;
}

int octmc_lbfgs_push(octmc_lbfgs* h, const double* s, const double* y) {
  if (!h || !s || !y) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    CK(cudaMemcpyAsync(h->S[h->spare], s, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->Y[h->spare], y, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->st));
    return h->prepare(nullptr, true);
  });
}

int octmc_lbfgs_direction(octmc_lbfgs* h, const double* g, double* dir, double* gtd) {
  if (!h || !g || !dir) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    h->prepare(g, false);
    const double v = h->direction(g, dir);
    CK(cudaStreamSynchronize(h->st));
    if (gtd) *gtd = v;
    return OCTMC_OK;
  });
}

int octmc_lbfgs_reset(octmc_lbfgs* h) {
  if (!h) return OCTMC_ERR_INVALID_ARG;
  h->reset();
  return OCTMC_OK;
}

int octmc_profile_enable(octmc_problem* p, int enable) {
  if (!p) return OCTMC_ERR_INVALID_ARG;
  return guarded([&] {
    if (enable && !p->ev0) {
      CK(cudaEventCreate(&p->ev0));
      CK(cudaEventCreate(&p->ev1));
    }
    p->profile = enable != 0;
    p->prof_ms = 0.0;
    p->prof_count = 0;
    p->prof_pending = false;
    return OCTMC_OK;
  });
}

int octmc_profile_read(octmc_problem* p, double* total_ms, long long* launches) {
  if (!p) return OCTMC_ERR_INVALID_ARG;
  if (total_ms) *total_ms = p->prof_ms;
  if (launches) *launches = p->prof_count;
  return OCTMC_OK;
}

int64_t octmc_estimate_bytes(const octmc_desc* desc) {
  if (!desc || desc->w < 1 || desc->h < 1 || desc->d < 1) return -1;
  return estimate_bytes_impl(*desc);
}

int octmc_server_create(int64_t budget_bytes, int max_slots, void* stream, octmc_server** out) {
  if (!out || budget_bytes <= 0 || max_slots < 1) return OCTMC_ERR_INVALID_ARG;
  *out = nullptr;
  octmc_server* s = new (std::nothrow) octmc_server();
  if (!s) return OCTMC_ERR_OOM;
  s->st = (cudaStream_t)stream;
  s->budget = budget_bytes;
  s->max_slots = std::min(max_slots, 1 << 16);
  const int rc = guarded([&] {
    check_device();
    return OCTMC_OK;
  });
  if (rc != OCTMC_OK) {
    delete s;
    return rc;
  }
  *out = s;
  return OCTMC_OK;
}

void octmc_server_destroy(octmc_server* s) { delete s; }

int octmc_server_submit(octmc_server* s, const octmc_desc* desc, int64_t* ticket) {
  if (!s || !desc || !ticket) return OCTMC_ERR_INVALID_ARG;
  const octmc_desc& D = *desc;
  if (D.w < 1 || D.h < 1 || D.d < 1 || !D.sx || !D.sy || !D.tx || !D.ty || (D.ax == nullptr) != (D.ay == nullptr) ||
      D.levels < 1 || D.levels > 16 || D.lbfgs_m < 1 || D.lbfgs_m > 32 || D.max_ls < 1 || D.max_iter < 0 ||
      (D.loss != OCTMC_LOSS_PSEUDO_HUBER && D.loss != OCTMC_LOSS_SSD) ||
      (D.storage != OCTMC_F32 && D.storage != OCTMC_BF16 && D.storage != OCTMC_F16) || !(D.eps_h > 0) ||
      !(D.eps_r > 0) || !(D.alpha >= 0) || !(D.delta0 >= 0))
    return OCTMC_ERR_INVALID_ARG;
  auto r = std::make_shared<octmc_server::Req>();
  r->ticket = s->next_ticket++;
  r->desc = D;
  // served solves run concurrently on their own streams: a cooperative grid
  // of one of them would wait for SMs that another holds
  r->desc.persistent_ascans = 0;
  r->bytes = estimate_bytes_impl(D);
  if (r->bytes > s->budget) return OCTMC_ERR_OOM;  // could never be admitted
  s->queue.push_back(r);
  s->all[r->ticket] = r;
  *ticket = r->ticket;
  return OCTMC_OK;
}

int octmc_server_step(octmc_server* s, int* active, int* queued) {
  if (!s) return OCTMC_ERR_INVALID_ARG;
  const int rc = guarded([&] {
    s->step();
    return OCTMC_OK;
  });
  if (active) *active = (int)s->active.size();
  if (queued) *queued = (int)s->queue.size();
  return rc;
}

int octmc_server_state(const octmc_server* s, int64_t ticket, int* state) {
  if (!s || !state) return OCTMC_ERR_INVALID_ARG;
  auto it = s->all.find(ticket);
  *state = (it == s->all.end()) ? OCTMC_REQ_UNKNOWN : it->second->state;
  return OCTMC_OK;
}

int octmc_server_poll(octmc_server* s, int64_t ticket, int* state, double* disp_out, octmc_stats* stats, int max_stats,
                      int* req_rc) {
  if (!s || !state) return OCTMC_ERR_INVALID_ARG;
  auto it = s->all.find(ticket);
  if (it == s->all.end()) {
    *state = OCTMC_REQ_UNKNOWN;
    return OCTMC_OK;
  }
  std::shared_ptr<octmc_server::Req> rp = it->second;
  octmc_server::Req& r = *rp;
  *state = r.state;
  if (r.state != OCTMC_REQ_DONE) return OCTMC_OK;
  const int rc = guarded([&] {
    if (disp_out && r.result) {
      if (r.done) CK(cudaStreamWaitEvent(s->st, r.done, 0));
      CK(cudaMemcpyAsync(disp_out, r.result, sizeof(double) * 6 * r.desc.w * r.desc.h, cudaMemcpyDeviceToDevice,
                         s->st));
      CK(cudaStreamSynchronize(s->st));
    }
    if (stats)
      for (int k = 0; k < max_stats && k < (int)r.stats.size(); k++) stats[k] = r.stats[k];
    return OCTMC_OK;
  });
  if (req_rc) *req_rc = r.rc;
  s->all.erase(it);
  s->release(rp);
  return rc;
}

int octmc_barrier_selftest(int extra) {
  if (extra < 0 || extra > 1) return OCTMC_ERR_INVALID_ARG;
  unsigned* bar = nullptr;
  if (cudaMalloc(&bar, 4 * sizeof(unsigned)) != cudaSuccess) return OCTMC_ERR_OOM;
  int rc = OCTMC_OK;
  int err = 0;
  if (cudaMemset(bar, 0, 4 * sizeof(unsigned)) != cudaSuccess ||
      launch_barrier_probe(bar, reinterpret_cast<int*>(bar + 2), extra, 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&err, bar + 2, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    rc = OCTMC_ERR_CUDA;
  } else if (err) {
    rc = OCTMC_ERR_TIMEOUT;
  }
  cudaFree(bar);
  return rc;
}

const char* octmc_status_string(int code) {
  switch (code) {
    case OCTMC_OK: return "ok";
    case OCTMC_NOT_CONVERGED: return "not converged (iteration cap)";
    case OCTMC_ERR_INVALID_ARG: return "invalid argument";
    case OCTMC_ERR_OOM: return "out of device memory";
    case OCTMC_ERR_CUDA: return "CUDA error";
    case OCTMC_ERR_NONFINITE: return "objective is not finite";
    case OCTMC_ERR_TIMEOUT: return "device wait timed out";
    case OCTMC_ERR_UNSUPPORTED: return "unsupported (needs an sm_103a device / dtype not built)";
    case OCTMC_ERR_SCRATCH_LIMIT: return "grid larger than the static scratch of octmc_data_term_static";
    default: return "unknown status";
  }
}

}  // extern "C"
