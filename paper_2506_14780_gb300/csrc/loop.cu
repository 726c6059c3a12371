// Device-side loop control for CUDA-graph while loops: the iteration loops of
// Algorithm 4.1 and of the mode computation run as conditional while nodes, so
// the host enqueues a whole continuation level (or a whole solve) and never
// polls.  Every body ends with one of these single-thread kernels; each loop is
// hard-capped by State::body_cap body executions so that it always terminates.
#include "eot_device.cuh"
#include "eot_internal.h"

namespace eotk {

// which = 0: Sinkhorn / SK-NR loop (State::done), 1: mode computation loop.
__global__ void loop_ctl_kernel(cudaGraphConditionalHandle h, State* st, int which, int use_cond) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->body_runs += 1;
  bool cont = which == 0 ? (st->done == 0) : (st->eig_done == 0);
  if (cont && st->body_runs >= st->body_cap) {
    cont = false;
    if (which == 0) st->done = 4;
    else st->eig_done = 4;
  }
  if (use_cond) cudaGraphSetConditional(h, cont ? 1u : 0u);
}

// Convergence bookkeeping of the mode computation after a Rayleigh-Ritz step.
// A residual that is not a finite number (the block broke down) stops the
// loop as not converged.
__global__ void eig_ctl_kernel(State* st, const double* resid, const int* fail) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->eig_iter += 1;
  st->eig_resid = *resid;
  if (*fail) { st->eig_fail += 1; }
  if (*resid <= st->eig_tol) st->eig_done = 1;
  else if (st->eig_iter >= st->eig_max_iter || !isfinite(*resid)) st->eig_done = 2;
}

// Level set-up: write the level's eps-dependent constants into the problem and
// reset the iteration state.  One thread.
__global__ void level_setup_kernel(Prob* P, double eps, float k2, double tol, int max_iter,
                                   int body_cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  P->eps = eps;
  P->k2 = k2;
  P->k2lo = (float)(1.0 / (eps * 0.6931471805599453) - (double)k2);
  State* st = P->st;
  st->iter = 0;
  st->done = 0;
  st->nr_acc = 0;
  st->nr_rej = 0;
  st->nr_ok = 0;
  st->tol = tol;
  st->max_iter = max_iter;
  st->numeric = 0;
  st->body_runs = 0;
  st->body_cap = body_cap;
  st->stall_l1 = 1e300;
  st->stall_at = P->stall_window;
}

__global__ void eig_setup_kernel(State* st, double tol, int max_iter, int body_cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->eig_iter = 0;
  st->eig_done = 0;
  st->eig_tol = tol;
  st->eig_max_iter = max_iter;
  st->eig_fail = 0;
  st->eig_resid = 0.0;
  st->body_runs = 0;
  st->body_cap = body_cap;
}

}  // namespace eotk

namespace eotk {

// End of a level: copy the current f and g into buffer 0 and refresh their
// split arrays at the level's eps (the modes and the next level start there).
__global__ void normalize_buffers_kernel(Prob* PP) {
  const Prob& P = *PP;
  const State* st = P.st;
  const int cf = st->cur_f, cg = st->cur_g;
  const int len = max(P.n, P.m);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
    double hi;
    float lo;
    if (i < P.n) {
      const double v = P.f[cf][i];
      P.f[0][i] = v;
      if (P.fA64[0]) P.fA64[0][i] = v + P.eps * P.loga[i];
      split_grid(v + P.eps * P.loga[i], P.qscale, P.qinv, hi, lo);
      P.rs[0].A[i] = (float)(hi + (double)P.M);
      P.rs[0].AL[i] = lo;
      split_grid(v, P.qscale, P.qinv, hi, lo);
      P.rs[0].K[i] = (float)((double)P.M - hi);
      P.rs[0].KL[i] = lo;
    }
    if (i < P.m) {
      const double v = P.g[cg][i];
      P.g[0][i] = v;
      if (P.gA64[0]) P.gA64[0][i] = v + P.eps * P.logb[i];
      split_grid(v + P.eps * P.logb[i], P.qscale, P.qinv, hi, lo);
      P.cs[0].A[i] = (float)(hi + (double)P.M);
      P.cs[0].AL[i] = lo;
      split_grid(v, P.qscale, P.qinv, hi, lo);
      P.cs[0].K[i] = (float)((double)P.M - hi);
      P.cs[0].KL[i] = lo;
    }
  }
}

__global__ void reset_buffers_kernel(State* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->cur_f = 0;
    st->cur_g = 0;
  }
}

}  // namespace eotk
