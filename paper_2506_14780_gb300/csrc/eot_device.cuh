// Device-side building blocks shared by the pass kernels.
//
// Exponent formation.  Every O(nm) pass evaluates terms
//     x_ij = (u_i + s_j - C_ij) / eps
// where u (per reduction index) and s (per output index) are float64
// potentials (already including eps * log(weight) where the transform needs it)
// and C_ij is the float32 cost.  Near a Sinkhorn fixed point the dominant terms
// have x_ij in [-30, 0], while u_i, s_j and C_ij are O(1): forming u + s - C in
// float32 would lose ~1e-7 absolute, i.e. ~1e-4 in x at eps = 1e-3.  The kernels
// instead split every potential p into
//     p = pH + pL,  pH on the grid 2^-q (exact in float32),  |pL| <= 2^-(q+1),
// and round C_ij to the same grid with one addition of a "magic" constant
// M = 1.5 * 2^(23-q) (all values stay inside the binade [2^(23-q), 2^(24-q)),
// whose float32 spacing is exactly 2^-q):
//     r  = C + (M - sH)         = (M - sH) + h,      h = C rounded to the grid
//     tH = (uH + M) - r         = uH + sH - h        (exact: same binade, Sterbenz)
//     h  = r - (M - sH),  l = C - h                  (both exact)
//     x * eps = (tH - l) + uL + sL
// so the only rounding errors are those of the last two additions, relative to
// |x * eps| itself.  The division by eps is a multiplication by log2(e)/eps
// folded into the exp2 argument together with sL.  Validity needs
// |pH| + |C| < 2^(22-q); the host picks q from the cost range.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace eotk {

// Programmatic dependent launch.  pdl_wait (griddepcontrol.wait) returns once
// the preceding kernel of the stream has completed and its memory operations
// are visible (at once when the kernel was not launched as a dependent);
// pdl_trigger lets the next kernel launch (its CTAs then wait in pdl_wait).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Entry of a kernel launched with launch_pdl: nothing the preceding kernels
// write is touched before it.
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_trigger();
}


constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
// Re-centring threshold of the running log-sum-exp (log2 units).
constexpr float kRecenter = 64.0f;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 2^(p + q) for the evaluation passes that verify a result: p a float32
// exponent (log2 units), q a small correction carried beside it (|q| < 1/4;
// the rounding error of p and the low parts of the potentials).  Range
// reduction p = n + f with n = rint(p) (f exact), x = (f + q) ln 2, and the
// Taylor series of e^x to degree 7 (|x| < 0.53: truncation below 1e-7, mostly
// below 1e-8), Horner in float32 with round-to-nearest, so that its rounding
// errors average out over a sum.  Two reasons for not using the iteration's
// arithmetic here: the hardware approximation ex2.approx is biased by a few
// 1e-8 relative with the same sign for every term (measured: -2e-8 to -5e-8
// for p in [-1, 0] to [-30, 0]), and an evaluation that repeated the
// iteration's rounding of each exponent would not see that rounding's effect
// on the marginals; either blind spot hides ~1e-7 of L1, a tenth of 1e-6.
__device__ __forceinline__ float ex2_pq(float p, float q) {
  if (!(p >= -126.f)) return 0.f;   // -inf (masked terms) and results below the normal range
  const float n = fminf(rintf(p), 127.f), x = ((p - n) + q) * 0.6931471805599453f;
  float r = 1.f / 5040.f;
  r = fmaf(r, x, 1.f / 720.f);
  r = fmaf(r, x, 1.f / 120.f);
  r = fmaf(r, x, 1.f / 24.f);
  r = fmaf(r, x, 1.f / 6.f);
  r = fmaf(r, x, 0.5f);
  r = fmaf(r, x, 1.f);
  r = fmaf(r, x, 1.f);
  return r * __int_as_float(((int)n + 127) << 23);   // exact scaling by 2^n
}

// The exact part of the exponent (see the header comment).
//   C: cost, K: M - sH (output-side shift), A: uH + M (reduction-side), returns
//   tH - l ; the caller adds uL and scales.
__device__ __forceinline__ float split_exponent(float C, float K, float A) {
  float r = __fadd_rn(C, K);
  float tH = __fsub_rn(A, r);
  float h = __fsub_rn(r, K);
  float l = __fsub_rn(C, h);
  return __fsub_rn(tH, l);
}

// Running (reference, sum) state of a log-sum-exp in log2 units:
//   S = sum_k 2^(y_k - ref); ref is re-centred when the running maximum leaves
//   [-kRecenter, kRecenter] around it, which keeps every term and the sum finite.
struct Lse2 {
  float ref;   // reference point (log2 units)
  float run;   // running max of (y - ref)
  float S;
  __device__ __forceinline__ void init() { ref = 0.f; run = -INFINITY; S = 0.f; }
};

// Scale by 2^k (k an integer held in a float): exact, underflows to 0.
__device__ __forceinline__ float scale2(float x, float k) {
  return ldexpf(x, (int)fmaxf(fminf(k, 300.f), -300.f));
}

// Combine two (ref, S) partial states: result in state a.  References are
// integers (log2 units), so the rescaling is an exact power of two.
__device__ __forceinline__ void lse2_merge(float& ra, float& Sa, float rb, float Sb) {
  if (Sb == 0.f) return;
  if (Sa == 0.f) { ra = rb; Sa = Sb; return; }
  if (ra == rb) { Sa += Sb; return; }
  if (ra > rb) { Sa += scale2(Sb, rb - ra); }
  else { Sa = scale2(Sa, ra - rb) + Sb; ra = rb; }
}

// Warp-wide sum of a double.
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Natural log of a positive float64 sum S: log1p of the exact S - 1 near 1 (so
// that a marginal ratio close to one keeps its relative precision), log of S
// otherwise (S - 1 would lose it when S << 1).
__device__ __forceinline__ float log_sum(double S) {
  return (S > 0.5 && S < 2.0) ? log1pf((float)(S - 1.0)) : logf((float)S);
}

// Split a float64 value into (grid-aligned hi, float32 lo) on the 2^-q grid.
__device__ __forceinline__ void split_grid(double x, double scale /*2^q*/, double inv /*2^-q*/,
                                           double& hi, float& lo) {
  hi = rint(x * scale) * inv;
  lo = (float)(x - hi);
}

}  // namespace eotk
