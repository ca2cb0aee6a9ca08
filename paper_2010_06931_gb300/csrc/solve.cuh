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

// The controller fields are read once (independent loads) and written back
// once: this runs in a single thread on state in global memory, where every
// dependent access would cost a round trip to L2.
//
// ft, dgt: f and grad . dir at the trial; gmaxt: max |grad| at the trial.
// Once a new iterate is taken (the start point, or an accepted step) the
// stopping tests run here: 3 iterations in a row with relative decrease
// below ftol (status 0), max_iter iterations (status 1), max |grad| <= gtol
// at the new iterate (status 0).  S->branch asks for the accepted-step work
// (history and direction) when the level goes on from a new iterate or a
// retry.
__device__ __forceinline__ void ls_decide_state(SolveState* S, double ft, double dgt, double gmaxt) {
  const int mode0 = S->mode, max_ls = S->max_ls, max_evals = S->max_evals, k0 = S->k, max_iter = S->max_iter;
  int ls = S->ls, evals = S->evals + 1, have_lo = S->have_lo, retried = S->retried;
  int iters = S->iters, small = S->small, status = S->status, done = S->done, mode = mode0, k = k0;
  double f = S->f, fb = S->fb, a = S->a, lo = S->lo, hi = S->hi, gmaxb = S->gmaxb;
  const double dg0 = S->dg0, ftol = S->ftol, gtol = S->gtol;
  int save_best = 0, restore_best = 0, branch = 0, moved = 0;
  double ftn = ft, gmax_new = gmaxt;
  if (mode0 == kModeInit) {
    f = ft;
    branch = 1;
    moved = 1;
  } else {
    ls++;
    const double at = a;
    bool accepted = false;
    if (!(ft <= f + 1e-4 * at * dg0)) {
      hi = at;
      a = 0.5 * (lo + hi);
    } else if (dgt < 0.9 * dg0) {
      lo = at;
      have_lo = 1;
      fb = ft;
      gmaxb = gmaxt;
      save_best = 1;
      a = isinf(hi) ? 2.0 * at : 0.5 * (lo + hi);
    } else {
      accepted = true;
    }
    if (!accepted && ls < max_ls && evals < max_evals) {
      branch = 0;  // next trial with the new step
    } else {
      if (!accepted) {
        if (have_lo) {
          restore_best = 1;
          ftn = fb;
          gmax_new = gmaxb;
          accepted = true;
        } else if (k > 0 && !retried) {
          k = 0;  // drop the history, retry from -g
          retried = 1;
          mode = kModeRetry;
          branch = 1;
        } else {
          status = 2;
          done = 1;
        }
      }
      if (accepted) {
        retried = 0;
        const double rel = (f - ftn) / fmax(fmax(fabs(f), fabs(ftn)), 1.0);
        f = ftn;
        iters++;
        small = (rel < ftol) ? small + 1 : 0;
        mode = kModeAccept;
        branch = 1;
        moved = 1;
      }
    }
  }
  if (moved && !done) {
    if (mode == kModeAccept && small >= 3) {
      status = 0;
      done = 1;
    } else if (iters >= max_iter) {
      status = 1;
      done = 1;
    } else if (gmax_new <= gtol) {
      status = 0;
      done = 1;
    }
  }
  if (evals >= max_evals && !done && branch == 0) {
    status = 2;
    done = 1;
  }
  if (done) branch = 0;  // nothing more to prepare: the level ends
  S->save_best = save_best;
  S->restore_best = restore_best;
  S->moved = moved;
  S->evals = evals;
  S->ls = ls;
  S->have_lo = have_lo;
  S->retried = retried;
  S->iters = iters;
  S->small = small;
  S->status = status;
  S->done = done;
  S->mode = mode;
  S->k = k;
  S->f = f;
  S->ft = ftn;
  S->fb = fb;
  S->gmaxb = gmaxb;
  S->a = a;
  S->lo = lo;
  S->hi = hi;
  S->branch = branch;
}

// The level loop goes on while the level is not done (hard cap on evaluations).
__device__ __forceinline__ bool ls_more(const SolveState* S) { return !S->done && S->evals < S->max_evals + 2; }

// The decision inside the solve graph: the state update, then the IF node's
// condition (the accepted-step branch) and the WHILE node's (the loop).
__device__ __forceinline__ void ls_decide(SolveState* S, double ft, double dgt, double gmaxt,
                                          cudaGraphConditionalHandle h_branch,
                                          cudaGraphConditionalHandle h_while) {
  ls_decide_state(S, ft, dgt, gmaxt);
  cudaGraphSetConditional(h_branch, S->branch ? 1u : 0u);
  cudaGraphSetConditional(h_while, ls_more(S) ? 1u : 0u);
}

}  // namespace octmc
