// Per-index finish and grid-final step shared by the log-sum-exp pass kernels
// (the striped passes in passes.cu and the staged stream passes in stream.cu).
#pragma once
#include "eot_device.cuh"
#include "eot_internal.h"

namespace eotk {

// ---------------------------------------------------------------------------
// Finish one index from its merged (R, S): new potential, split arrays, the
// index's contributions (w |expm1 L|, w L, w out) to the scalars.  The index's
// shift, weight and log-weight are passed as values (they may be loaded ahead).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finish_index_v(float R, double S, int idx, const Prob& P,
                                               double sh, double wi, double logwi,
                                               double* __restrict__ out, Split so,
                                               float* __restrict__ Lout, double acc[3],
                                               int* numeric) {
  // the log-ratio in float64: far from the shift (|L| large) a float32 L
  // would move the output by eps |L| 2^-24
  double Ld = (double)R * 0.6931471805599453 + (double)log_sum(S);
  double o = sh - P.eps * Ld;
  if (!isfinite(o) || !(S > 0.0) || fabs(o) > P.pot_bound) {
    atomicAdd(numeric, 1);
    o = sh;
    Ld = 0.0;
  }
  const float L = (float)Ld;
  if (out) out[idx] = o;
  if (Lout) Lout[idx] = L;
  if (so.A && so.nrm) {
    double hi;
    float lo;
    split_grid((double)P.k2 * (o - so.nrm[idx]), P.qscale, P.qinv, hi, lo);
    so.A[idx] = (float)wi;
    so.AL[idx] = 0.f;
    so.K[idx] = (float)hi;
    so.KL[idx] = lo;
  } else if (so.A) {
    double hi;
    float lo;
    split_grid(o + P.eps * logwi, P.qscale, P.qinv, hi, lo);
    so.A[idx] = (float)(hi + (double)P.M);
    so.AL[idx] = lo;
    split_grid(o, P.qscale, P.qinv, hi, lo);
    so.K[idx] = (float)((double)P.M - hi);
    so.KL[idx] = lo;
  }
  acc[0] = wi * (double)fabsf(expm1f(L));
  acc[1] = wi * Ld;
  acc[2] = wi * o;
}

__device__ __forceinline__ void finish_index(float R, double S, int idx, const Prob& P,
                                             const double* __restrict__ shift,
                                             const double* __restrict__ w,
                                             const double* __restrict__ logw,
                                             double* __restrict__ out, Split so,
                                             float* __restrict__ Lout, double acc[3],
                                             int* numeric) {
  finish_index_v(R, S, idx, P, shift[idx], w[idx], so.A ? logw[idx] : 0.0, out, so, Lout, acc,
                 numeric);
}

// Block-wide deterministic sum of 3 doubles; result valid in thread 0.
__device__ __forceinline__ void block_sum3(double v[3], double* sh /*[3*8]*/) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double x = warp_sum_d(v[k]);
    if (lane == 0) sh[k * 8 + wid] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      double t = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[k * 8 + i];
      v[k] = t;
    }
  }
  __syncthreads();
}

// Grid-final step shared by both passes.  Called by one thread with the sums.
__device__ inline void final_step(const Prob& P, int mode, const double t[3], int dst) {
  State* st = P.st;
  st->sum_wL = t[1];
  st->sum_wout = t[2];
  if (st->numeric > 0 && mode != MODE_PLAIN && mode != MODE_EVAL) {
    st->done = 3;
    return;
  }
  switch (mode) {
    case MODE_SK_ROW:
      st->l1_row = t[0];
      st->sum_af = t[2];
      break;
    case MODE_TRIAL: {
      // Q_semi(f') - Q_semi(f_k) = <V Delta, a> + <h' - h, b>,  h' - h = -eps L
      const double dq = st->dot_vd_a - P.eps * t[1];
      st->dq = dq;
      trace_trial(P, st, dq, dq > 0.0 ? 1 : 0);
      if (dq > 0.0) {
        st->nr_acc += 1;
        st->cur_f = 1 - st->cur_f;
        st->cur_g = (st->cur_g + 2) % 3;
      } else {
        st->nr_rej += 1;
        st->cur_g = (st->cur_g + 1) % 3;
      }
      break;
    }
    case MODE_SK_COL:
      st->l1_col = t[0];
      st->qsemi = st->sum_af + t[2];   // Q_semi(f_k) = <f_k, a> + <f_k^{C,eps}, b>
      st->iter += 1;
      trace_test(P, st, st->iter, t[0], st->qsemi);
      st->done = stop_code(st, t[0], st->iter, st->tol, st->max_iter, P.stall_window);
      if (!st->done) st->cur_g = dst;
      break;
    case MODE_EVAL:
      st->l1_col = t[0];
      break;
    case MODE_G_INIT:
      st->cur_g = dst;
      break;
    default:
      st->l1_col = t[0];
      break;
  }
}

}  // namespace eotk
