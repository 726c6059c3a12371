// Deterministic cross-segment reductions used by the last-arriving CTA of a
// pass: the partial (reference, sum) states of every segment are loaded in
// parallel (several independent loads per thread in flight), merged in float64
// with exact power-of-two rescaling, and then combined across threads in a
// fixed order, so the result never depends on scheduling.
#pragma once
#include "eot_device.cuh"

namespace eotk {

// Merge a float partial (ref, sum) into a float64 running state.
__device__ __forceinline__ void merge_d(float& R, double& S, float r, float s) {
  if (!(s > 0.f)) return;
  if (S == 0.0) {
    R = r;
    S = (double)s;
  } else if (r == R) {
    S += (double)s;
  } else if (r < R) {
    S += ldexp((double)s, (int)fmaxf(r - R, -1000.f));
  } else {
    S = ldexp(S, (int)fmaxf(R - r, -1000.f)) + (double)s;
    R = r;
  }
}

__device__ __forceinline__ void merge_dd(float& R, double& S, float r, double s) {
  if (!(s > 0.0)) return;
  if (S == 0.0) {
    R = r;
    S = s;
  } else if (r == R) {
    S += s;
  } else if (r < R) {
    S += ldexp(s, (int)fmaxf(r - R, -1000.f));
  } else {
    S = ldexp(S, (int)fmaxf(R - r, -1000.f)) + s;
    R = r;
  }
}

// Thread-local merge of segments seg = first, first + step, ... of index idx
// (part laid out [segment][stride]); four loads in flight per round.
__device__ __forceinline__ void merge_segments(const float2* __restrict__ part, int nseg, int stride,
                                               int idx, int first, int step, float& R, double& S) {
  R = -INFINITY;
  S = 0.0;
  for (int s0 = first; s0 < nseg; s0 += 4 * step) {
    float2 p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s = s0 + q * step;
      p[q] = s < nseg ? __ldcg(&part[(size_t)s * stride + idx]) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) merge_d(R, S, p[q].x, p[q].y);
  }
}

// Merge the (ref, sum) heads of records part[(s * stride + idx) * width + {0,1}]
// over all segments s, four loads in flight per round.
__device__ __forceinline__ void merge_segments_k(const float* __restrict__ part, int nseg,
                                                 int stride, int width, int idx, float& R,
                                                 double& S) {
  R = -INFINITY;
  S = 0.0;
  for (int s0 = 0; s0 < nseg; s0 += 4) {
    float pr[4], ps[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s = s0 + q;
      const float* src = part + ((size_t)s * stride + idx) * width;
      pr[q] = s < nseg ? __ldcg(src) : 0.f;
      ps[q] = s < nseg ? __ldcg(src + 1) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) merge_d(R, S, pr[q], ps[q]);
  }
}

// Sum of nblk x 3 block accumulators (stride 4) by all threads of one CTA, in a
// fixed order; result valid in every thread.  Uses sh[3 * 8].
__device__ __forceinline__ void grid_sum3(const double* __restrict__ acc, int nblk, double out[3],
                                          double* sh) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    v[0] += __ldcg(&acc[b * 4 + 0]);
    v[1] += __ldcg(&acc[b * 4 + 1]);
    v[2] += __ldcg(&acc[b * 4 + 2]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k * 8 + wid] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[k * 8 + w];
    out[k] = t;
  }
  __syncthreads();
}

}  // namespace eotk
