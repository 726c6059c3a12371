// Cost construction and whole-vector reductions.
//
//  * cost kernels: C_ij = ||x_i - y_j||^2 (Sec. 2 and Sec. 5: squared Euclidean
//    cost between the samples) in float64, summed over the coordinates in order,
//    optionally divided by max_ij C_ij, rounded once to float32;
//  * cost_stats: max |C_ij| and the number of non-finite entries of a given C;
//  * final_eval: the scores of the returned potentials (marginal errors, Eq.
//    def_Q value, duality gap) and the gauge normalisation <f,a> = <g,b>
//    (Sec. 2: the dual is invariant under (f, g) + c (1, -1)).
#include "eot_device.cuh"
#include "eot_internal.h"

namespace eotk {

__device__ __forceinline__ double sqdist(const float* __restrict__ x, const float* __restrict__ y,
                                         int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    const double t = __dsub_rn((double)x[k], (double)y[k]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}

// max over all entries (non-negative doubles compare like their bit patterns)
__global__ void cost_max_kernel(int n, int m, int d, const float* __restrict__ X,
                                const float* __restrict__ Y, unsigned long long* __restrict__ out) {
  double mx = 0.0;
  const size_t total = (size_t)n * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e - (size_t)i * m);
    mx = fmax(mx, sqdist(X + (size_t)i * d, Y + (size_t)j * d, d));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

__global__ void cost_fill_kernel(int n, int m, int d, const float* __restrict__ X,
                                 const float* __restrict__ Y,
                                 const unsigned long long* __restrict__ cmax_bits, int normalize,
                                 float* __restrict__ C) {
  const double cmax = __longlong_as_double((long long)*cmax_bits);
  const size_t total = (size_t)n * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e - (size_t)i * m);
    double v = sqdist(X + (size_t)i * d, Y + (size_t)j * d, d);
    if (normalize && cmax > 0.0) v = __ddiv_rn(v, cmax);
    C[e] = __double2float_rn(v);
  }
}

// Scale a given cost by 1 / max (normalisation of a user-supplied C).
__global__ void cost_scale_kernel(size_t total, const float* __restrict__ Cin, double cmax,
                                  float* __restrict__ Cout) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    Cout[e] = __double2float_rn(__ddiv_rn((double)Cin[e], cmax));
}

// max |C| as float bits and the count of non-finite entries
__global__ void cost_stats_kernel(size_t total, const float* __restrict__ C,
                                  unsigned* __restrict__ maxbits, unsigned* __restrict__ bad) {
  float mx = 0.f;
  unsigned nb = 0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const float v = C[e];
    if (!isfinite(v)) ++nb;
    else mx = fmaxf(mx, fabsf(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(maxbits, __float_as_uint(mx));
    if (nb) atomicAdd(bad, nb);
  }
}

// Float64 variant of the same statistics (FP64 cost path).
__global__ void cost_stats_f64_kernel(size_t total, const double* __restrict__ C,
                                      unsigned long long* __restrict__ maxbits,
                                      unsigned* __restrict__ bad) {
  double mx = 0.0;
  unsigned nb = 0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const double v = C[e];
    if (!isfinite(v)) ++nb;
    else mx = fmax(mx, fabs(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(maxbits, (unsigned long long)__double_as_longlong(mx));
    if (nb) atomicAdd(bad, nb);
  }
}

// Weights: w <- w / sum(w), logw = log(w); flags non-positive / non-finite.
// One CTA (deterministic sum).
__global__ void __launch_bounds__(256) weights_kernel(int len, const double* __restrict__ win,
                                                      double* __restrict__ w,
                                                      double* __restrict__ logw,
                                                      unsigned* __restrict__ bad, int normalize) {
  __shared__ double sh[8];
  __shared__ double s_tot;
  double s = 0.0;
  unsigned nb = 0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const double v = win[i];
    if (!(v > 0.0) || !isfinite(v)) ++nb;
    s += v;
  }
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  if (nb) atomicAdd(bad, nb);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += sh[k];
    s_tot = t;
  }
  __syncthreads();
  const double tot = normalize ? s_tot : 1.0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const double v = win[i] / tot;
    w[i] = v;
    logw[i] = log(v);
  }
}

// ---------------------------------------------------------------------------
// Final scores and gauge normalisation of (f, g) = (f[cur_f], g[cur_g]), using
// the marginal log-ratios Lrow, Lcol of pi(f, g) from two evaluation passes:
//   (pi 1)_i = a_i exp(Lrow_i),  (pi^T 1)_j = b_j exp(Lcol_j).
// out[0..7] = row_l1, col_l1, <f,a>, <g,b>, sum pi, q_dual, gap, shift c.
// One CTA; f_out, g_out receive the shifted potentials (device).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) final_eval_kernel(const Prob* __restrict__ PP,
                                                         double* __restrict__ f_out,
                                                         double* __restrict__ g_out,
                                                         double* __restrict__ out) {
  const Prob& P = *PP;
  const State* st = P.st;
  const double* f = P.f[st->cur_f];
  const double* g = P.g[st->cur_g];
  __shared__ double sh[8][8];
  __shared__ double tot[8];
  double v[6] = {0, 0, 0, 0, 0, 0};  // row_l1, col_l1, fa, gb, sumpi, gap_lin
  for (int i = threadIdx.x; i < P.n; i += blockDim.x) {
    const double e = (double)expm1f(P.Lrow[i]);
    const double ai = P.a[i];
    v[0] += ai * fabs(e);
    v[2] += ai * f[i];
    v[4] += ai * (1.0 + e);
    v[5] += ai * e * f[i];
  }
  for (int j = threadIdx.x; j < P.m; j += blockDim.x) {
    const double e = (double)expm1f(P.Lcol[j]);
    const double bj = P.b[j];
    v[1] += bj * fabs(e);
    v[3] += bj * g[j];
    v[5] += bj * e * g[j];
  }
  for (int k = 0; k < 6; ++k) {
    const double x = warp_sum_d(v[k]);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
    tot[threadIdx.x] = t;
  }
  __syncthreads();
  const double c = 0.5 * (tot[3] - tot[2]);
  for (int i = threadIdx.x; i < P.n; i += blockDim.x) f_out[i] = f[i] + c;
  for (int j = threadIdx.x; j < P.m; j += blockDim.x) g_out[j] = g[j] - c;
  if (threadIdx.x == 0) {
    out[0] = tot[0];
    out[1] = tot[1];
    out[2] = tot[2];
    out[3] = tot[3];
    out[4] = tot[4];
    out[5] = tot[2] + tot[3] - P.eps * (tot[4] - 1.0);   // Q_eps(f, g), Eq. def_Q
    out[6] = tot[5] + P.eps * (tot[4] - 1.0);            // <pi1-a,f>+<pi^T1-b,g>+eps(sum pi-1)
    out[7] = c;
  }
}

}  // namespace eotk

namespace eotk {

// Float64 cost (no rounding), optionally divided by the maximum.
__global__ void cost_fill64_kernel(int n, int m, int d, const float* __restrict__ X,
                                   const float* __restrict__ Y,
                                   const unsigned long long* __restrict__ cmax_bits, int normalize,
                                   double* __restrict__ C) {
  const double cmax = __longlong_as_double((long long)*cmax_bits);
  const size_t total = (size_t)n * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e - (size_t)i * m);
    double v = sqdist(X + (size_t)i * d, Y + (size_t)j * d, d);
    if (normalize && cmax > 0.0) v = __ddiv_rn(v, cmax);
    C[e] = v;
  }
}

// Optional in-place division of a float64 cost by its maximum, and the float32
// rounding used by the mode computation.
__global__ void cost64_finish_kernel(size_t total, double* __restrict__ C,
                                     const unsigned long long* __restrict__ cmax_bits,
                                     int normalize, float* __restrict__ Cf) {
  const double cmax = __longlong_as_double((long long)*cmax_bits);
  const bool scale = normalize && cmax > 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    double v = C[e];
    if (scale) {
      v = __ddiv_rn(v, cmax);
      C[e] = v;
    }
    Cf[e] = __double2float_rn(v);
  }
}

}  // namespace eotk
