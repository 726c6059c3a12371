// Cost construction and whole-vector reductions.
//
//  * cost kernels: C_ij = ||x_i - y_j||^2 (Sec. 2 and Sec. 5: squared Euclidean
//    cost between the samples) in float64, summed over the coordinates in order,
//    optionally divided by max_ij C_ij, rounded once to float32;
//  * cost_stats: max |C_ij| and the number of non-finite entries of a given C;
//  * final_eval: the scores of the returned potentials (marginal errors, Eq.
//    def_Q value, duality gap) and the gauge normalisation <f,a> = <g,b>
//    (Sec. 2: the dual is invariant under (f, g) + c (1, -1)).
#include <algorithm>
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

// ---------------------------------------------------------------------------
// Tiled cost construction from points (rows of a tile staged in shared
// memory, threads over columns: no per-element index division).
// ---------------------------------------------------------------------------
constexpr int kCostRows = 32;

// float32 approximation of ||x_i - y_j||^2: relative error below
// (d + 3) 2^-24 (every term is non-negative).
__device__ __forceinline__ float sqdist_f(const float* __restrict__ x, const float* __restrict__ y,
                                          int d) {
  float s = 0.f;
  for (int k = 0; k < d; ++k) {
    const float t = x[k] - y[k];
    s = __fmaf_rn(t, t, s);
  }
  return s;
}

// Pass A of the exact maximum: max over the float32 approximations
// (non-negative floats compare like their bit patterns).
__global__ void __launch_bounds__(256) cost_maxf_kernel(int n, int m, int d,
                                                        const float* __restrict__ X,
                                                        const float* __restrict__ Y,
                                                        unsigned* __restrict__ fmax_bits) {
  extern __shared__ float sx[];   // [kCostRows][d]
  const int i0 = blockIdx.x * kCostRows, nr = min(kCostRows, n - i0);
  for (int e = threadIdx.x; e < nr * d; e += blockDim.x) sx[e] = X[(size_t)i0 * d + e];
  __syncthreads();
  float mx = 0.f;
  for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < m; j += gridDim.y * blockDim.x) {
    const float* y = Y + (size_t)j * d;
    for (int r = 0; r < nr; ++r) mx = fmaxf(mx, sqdist_f(sx + r * d, y, d));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(fmax_bits, __float_as_uint(mx));
}

// Pass B: the exact float64 distance of every candidate pair, those whose
// approximation lies within twice the approximation's error of the
// approximate maximum (the exact maximum is among them).
__global__ void __launch_bounds__(256) cost_maxx_kernel(int n, int m, int d,
                                                        const float* __restrict__ X,
                                                        const float* __restrict__ Y,
                                                        const unsigned* __restrict__ fmax_bits,
                                                        unsigned long long* __restrict__ out) {
  extern __shared__ float sx[];   // [kCostRows][d]
  const int i0 = blockIdx.x * kCostRows, nr = min(kCostRows, n - i0);
  for (int e = threadIdx.x; e < nr * d; e += blockDim.x) sx[e] = X[(size_t)i0 * d + e];
  __syncthreads();
  const float fm = __uint_as_float(*fmax_bits);
  const float thr = fm * (1.f - 2.f * (float)(d + 4) * 1.1920929e-7f);
  double mx = 0.0;
  for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < m; j += gridDim.y * blockDim.x) {
    const float* y = Y + (size_t)j * d;
    for (int r = 0; r < nr; ++r)
      if (sqdist_f(sx + r * d, y, d) >= thr) mx = fmax(mx, sqdist(sx + r * d, y, d));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0)
    atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// RN32(RN64(v / cmax)) from rc = RN64(1 / cmax).  q = RN64(v rc) lies within
// 2 units in the last place of RN64(v / cmax) (|q - v / cmax| < 2 ulp); both
// round to the same float32 unless a float32 rounding midpoint is that close,
// i.e. unless the 29 bits of q below float32 precision are within 2 of
// 2^28 (or q is below the float32 normal range).  Only then is the quotient
// corrected once (Markstein's theorem: e = v - cmax q is exact by FMA and
// RN64(q + e rc) is the correctly rounded v / cmax).
__device__ __forceinline__ float round_quotient(double v, double cmax, double rc) {
  const double q = __dmul_rn(v, rc);
  const unsigned long long b = (unsigned long long)__double_as_longlong(q);
  const unsigned low = (unsigned)(b & 0x1FFFFFFFull);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex > 1023 - 126 && low - ((1u << 28) - 2u) > 4u) return __double2float_rn(q);
  const double e = fma(-q, cmax, v);
  return __double2float_rn(fma(e, rc, q));
}

// C_ij in float64, optionally divided by the maximum, rounded once to float32.
// The tile's rows are converted to float64 once (shared memory); points of up
// to 4 coordinates keep the column's point in float64 registers.
__global__ void __launch_bounds__(256) cost_fill2_kernel(int n, int m, int d,
                                                         const float* __restrict__ X,
                                                         const float* __restrict__ Y,
                                                         const unsigned long long* __restrict__ cmax_bits,
                                                         int normalize, float* __restrict__ C) {
  extern __shared__ double sxd[];   // [kCostRows][d]
  const int i0 = blockIdx.x * kCostRows, nr = min(kCostRows, n - i0);
  for (int e = threadIdx.x; e < nr * d; e += blockDim.x) sxd[e] = (double)X[(size_t)i0 * d + e];
  __syncthreads();
  const double cmax = __longlong_as_double((long long)*cmax_bits);
  const bool norm = normalize && cmax > 0.0;
  const double rc = norm ? 1.0 / cmax : 1.0;
  const bool small = d <= 4;
  for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < m; j += gridDim.y * blockDim.x) {
    const float* y = Y + (size_t)j * d;
    double yd[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) yd[k] = (small && k < d) ? (double)y[k] : 0.0;
    for (int r = 0; r < nr; ++r) {
      const double* x = sxd + r * d;
      double v;
      if (small) {
        // the same operations, in the same order, as sqdist
        const double t0 = __dsub_rn(x[0], yd[0]);
        v = __dmul_rn(t0, t0);
#pragma unroll
        for (int k = 1; k < 4; ++k) {
          if (k < d) {
            const double t = __dsub_rn(x[k], yd[k]);
            v = __dadd_rn(v, __dmul_rn(t, t));
          }
        }
      } else {
        v = 0.0;
        for (int k = 0; k < d; ++k) {
          const double t = __dsub_rn(x[k], (double)y[k]);
          v = __dadd_rn(v, __dmul_rn(t, t));
        }
      }
      C[(size_t)(i0 + r) * m + j] = norm ? round_quotient(v, cmax, rc) : __double2float_rn(v);
    }
  }
}

// Cost from points: the exact maximum (when wanted; into *cmax64, which the
// caller zeroed) and the cost (when C is given).  Wide points (more than 192
// coordinates) take the untiled kernels.
cudaError_t launch_cost_points(int n, int m, int d, const float* X, const float* Y, bool want_max,
                               int normalize, float* C, unsigned* fmax_bits,
                               unsigned long long* cmax64, cudaStream_t s) {
  const size_t sm = (size_t)kCostRows * d * sizeof(float);
  const size_t sm64 = (size_t)kCostRows * d * sizeof(double);   // the fill kernel's rows
  if (sm64 > 48 * 1024) {
    const size_t nm = (size_t)n * m;
    const int gb = (int)std::min<size_t>((nm + 255) / 256, 2048);
    if (want_max) cost_max_kernel<<<gb, 256, 0, s>>>(n, m, d, X, Y, cmax64);
    if (C) cost_fill_kernel<<<gb, 256, 0, s>>>(n, m, d, X, Y, cmax64, normalize, C);
    return cudaGetLastError();
  }
  const dim3 grid((n + kCostRows - 1) / kCostRows, std::min(16, (m + 255) / 256));
  if (want_max) {
    cudaError_t e = cudaMemsetAsync(fmax_bits, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cost_maxf_kernel<<<grid, 256, sm, s>>>(n, m, d, X, Y, fmax_bits);
    cost_maxx_kernel<<<grid, 256, sm, s>>>(n, m, d, X, Y, fmax_bits, cmax64);
  }
  if (C) cost_fill2_kernel<<<grid, 256, sm64, s>>>(n, m, d, X, Y, cmax64, normalize, C);
  return cudaGetLastError();
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
