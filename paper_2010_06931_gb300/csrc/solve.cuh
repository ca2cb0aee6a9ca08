// Line-search decision of the device-resident level solve (Ploner et al.,
// Sec. 2.1: "gradient-based L-BFGS solver"), run by one thread of the
// regulariser kernel's last block once the objective f(x + a dir) and
// grad(x + a dir) . dir of a trial are known.
//
// Weak-Wolfe bisection with c1 = 1e-4, c2 = 0.9: a trial that fails the
// Armijo test (or is not finite) halves the bracket; one that passes it but
// fails the curvature test raises the lower end (the best such point is
// kept; a doubles while there is no upper end); otherwise it is accepted.
// After max_ls trials the best Armijo point is taken; without one, the
// history is dropped and the step retried once from -g; then the level
// stops (status 2).  The same rules as the host-driven solver and the
// oracle's minimiser.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace octmc {

__device__ __forceinline__ void ls_decide(SolveState* S, double ft, double dgt, cudaGraphConditionalHandle h_branch) {
  S->save_best = 0;
  S->restore_best = 0;
  S->evals++;
  int branch = 0;
  if (S->mode == kModeInit) {
    S->f = ft;
    S->ft = ft;
    branch = 1;
  } else {
    S->ft = ft;
    S->ls++;
    const double a = S->a;
    bool accepted = false;
    if (!(ft <= S->f + 1e-4 * a * S->dg0)) {
      S->hi = a;
      S->a = 0.5 * (S->lo + S->hi);
    } else if (dgt < 0.9 * S->dg0) {
      S->lo = a;
      S->have_lo = 1;
      S->fb = ft;
      S->save_best = 1;
      S->a = isinf(S->hi) ? 2.0 * a : 0.5 * (S->lo + S->hi);
    } else {
      accepted = true;
    }
    if (!accepted && S->ls < S->max_ls && S->evals < S->max_evals) {
      branch = 0;  // next trial with the new step
    } else {
      if (!accepted) {
        if (S->have_lo) {
          S->restore_best = 1;
          S->ft = S->fb;
          accepted = true;
        } else if (S->k > 0 && !S->retried) {
          S->k = 0;  // drop the history, retry from -g
          S->retried = 1;
          S->mode = kModeRetry;
          branch = 1;
        } else {
          S->status = 2;
          S->done = 1;
        }
      }
      if (accepted) {
        S->retried = 0;
        const double fo = S->f, fn = S->ft;
        const double rel = (fo - fn) / fmax(fmax(fabs(fo), fabs(fn)), 1.0);
        S->f = fn;
        S->iters++;
        S->small = (rel < S->ftol) ? S->small + 1 : 0;
        S->mode = kModeAccept;
        branch = 1;
      }
    }
  }
  if (S->evals >= S->max_evals && !S->done && branch == 0) {
    S->status = 2;
    S->done = 1;
  }
  S->branch = branch;
  cudaGraphSetConditional(h_branch, branch ? 1u : 0u);
}

}  // namespace octmc
