// The coupling of a pair of potentials and its scalars (Eq. pi(f,g), Eq.
// primal_EOT):
//
//   P_ij = a_i b_j exp((f_i + g_j - C_ij) / eps),
//   <C, P>, sum P, and sum P log(P / (a b)) (the primal value is
//   <C, P> + eps KL(P | a x b) with that KL).
//
// At a solution P is the derivative of the optimal value with respect to C
// (envelope theorem: d Q_eps / d C_ij = a_i b_j exp((f_i + g_j - C_ij)/eps)).
// One CTA per row; the exponent is formed in float64 from the float64
// potentials and the float32 cost, its exponential in float64, the entry
// stored as float32.  The scalars are summed per row (fixed order) and then
// over the rows (fixed order): deterministic.
#include <algorithm>
#include "eot_device.cuh"
#include "eot_internal.h"

namespace eotk {

__global__ void __launch_bounds__(256) plan_row_kernel(int n, int m, const float* __restrict__ C,
                                                       const double* __restrict__ f,
                                                       const double* __restrict__ g,
                                                       const double* __restrict__ a,
                                                       const double* __restrict__ b, double eps,
                                                       float* __restrict__ P,
                                                       double* __restrict__ part) {
  __shared__ double red[3][8];
  const double inv = 1.0 / eps;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const double fi = f[i], ai = a[i];
    const float* Ci = C + (size_t)i * m;
    double sc = 0.0, sm = 0.0, sx = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const double c = (double)Ci[j];
      const double x = (fi + g[j] - c) * inv;
      const double p = ai * b[j] * exp(x);
      if (P) P[(size_t)i * m + j] = (float)p;
      sc += p * c;
      sm += p;
      sx += p * x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sc += __shfl_xor_sync(0xffffffffu, sc, o);
      sm += __shfl_xor_sync(0xffffffffu, sm, o);
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
      red[0][w] = sc;
      red[1][w] = sm;
      red[2][w] = sx;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double t = 0.0;
      for (int k = 0; k < 8; ++k) t += red[threadIdx.x][k];
      part[(size_t)i * 3 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// Sum of the n row records (one CTA; each thread a strided share in order,
// then the threads in order).
__global__ void __launch_bounds__(256) plan_sum_kernel(int n, const double* __restrict__ part,
                                                       double* __restrict__ out) {
  __shared__ double red[3][256];
  double s[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int k = 0; k < 3; ++k) s[k] += part[(size_t)i * 3 + k];
  for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int u = 0; u < (int)blockDim.x; ++u) t += red[threadIdx.x][u];
    out[threadIdx.x] = t;
  }
}

cudaError_t launch_plan(int n, int m, const float* C, const double* f, const double* g,
                        const double* a, const double* b, double eps, float* P, double* part,
                        double* out, int nsm, cudaStream_t s) {
  const int grid = std::max(1, std::min(n, 16 * nsm));
  plan_row_kernel<<<grid, 256, 0, s>>>(n, m, C, f, g, a, b, eps, P, part);
  plan_sum_kernel<<<1, 256, 0, s>>>(n, part, out);
  return cudaGetLastError();
}

}  // namespace eotk
