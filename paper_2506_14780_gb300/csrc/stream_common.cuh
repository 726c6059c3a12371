// Device helpers shared by the staged kernels (stream.cu, gram.cu): barriers
// of the 256 consumer threads (threads 0..255 of the CTA), mbarrier, bulk and
// tensor copies, acquire-release counters, programmatic dependent launch, the
// stream-K owner rule, lean float64 reductions and the running-reference rule
// of the log-sum-exp.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include "eot_device.cuh"
#include "eot_internal.h"
#include "tc.cuh"

namespace eotk {

constexpr int kStConsumers = 256;
constexpr float kStWindow = 64.f;

__device__ __forceinline__ void cons_sync() {
  asm volatile("bar.sync 1, 256;" ::: "memory");
}

// Barrier of the 256 consumer threads that also ORs a predicate over them, so
// that every consumer sees the same value.
__device__ __forceinline__ int cons_sync_or(int pred) {
  int out;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.s32 p, %1, 0;\nbar.red.or.pred q, 1, 256, p;\n"
      "selp.s32 %0, 1, 0, q;\n}"
      : "=r"(out)
      : "r"(pred)
      : "memory");
  return out;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive1(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bulk global -> shared copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Tiled tensor copy of the box at (x = column, y = row) of a 2-D tensor map;
// the whole box is counted on the mbarrier (out-of-range elements read as 0).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Arrival counter with acquire-release semantics at GPU scope: the release
// covers every write of the CTA ordered before it by a barrier (so only the
// counting thread needs it), the acquire makes the other arrivals' writes
// visible to the CTA after the next barrier.
__device__ __forceinline__ unsigned arrive_count(unsigned* p) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
  return old;
}

// CTA whose chunk holds tile t (chunks [floor(kT/G), floor((k+1)T/G)), G <= T).
__device__ __forceinline__ int st_owner(long long t, long long T, int G) {
  return (int)(((t + 1) * (long long)G - 1) / T);
}

// Float64 arithmetic is slow on this GPU (a small fraction of the float32
// rate), so the reductions below use as few float64 operations as a fixed
// summation order allows.

// Sum of three doubles held by the first `nact` consumer threads (a multiple
// of 32, the others hold zeros); valid in thread 0.
__device__ __forceinline__ void cons_sum3(double v[3], double* sh, int nact) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = nact >> 5;
  if (wid < nw) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double x = warp_sum_d(v[k]);
      if (lane == 0) sh[k * 8 + wid] = x;
    }
  }
  cons_sync();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += sh[k * 8 + w];
      v[k] = t;
    }
  }
}

// Sum of nblk per-block accumulators (stride 4) in a fixed order by warp 0;
// result valid in thread 0.
__device__ __forceinline__ void warp0_grid_sum3(const double* __restrict__ acc, int nblk,
                                                double out[3]) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += 32) {
    v[0] += __ldcg(&acc[b * 4 + 0]);
    v[1] += __ldcg(&acc[b * 4 + 1]);
    v[2] += __ldcg(&acc[b * 4 + 2]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) out[k] = warp_sum_d(v[k]);
}

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

// Compensated (Kahan) accumulation of a pair of running sums: S + x with the
// rounding error carried in c (the sum is S - c).  A long serial float32 sum
// would otherwise leave a relative error growing with the square root of the
// number of additions, which the L1 marginal test (a sum of absolute
// deviations) would read as a floor.
__device__ __forceinline__ void kahan_add2(float2& S, float2& c, float2 x) {
  const float2 m1 = f2(-1.f, -1.f);
  const float2 y = __ffma2_rn(c, m1, x);                 // x - c
  const float2 t = __fadd2_rn(S, y);
  c = __ffma2_rn(y, m1, __ffma2_rn(S, m1, t));           // (t - S) - y
  S = t;
}

// Fold the carried error into the sum (before a rescaling or a read-out).
__device__ __forceinline__ void kahan_fold2(float2& S, float2& c) {
  S = __ffma2_rn(c, f2(-1.f, -1.f), S);
  c = f2(0.f, 0.f);
}

__device__ __forceinline__ float2 ex2_2(float2 y) {
  return make_float2(ex2_approx(y.x), ex2_approx(y.y));
}

// Reference rule of a running sum (all values in log2 units).  The terms are
// formed as z = y - ref from the raw exponent y (relative to the output
// potential's shift), so a reference of exactly 0 keeps them exact.  The
// reference stays 0 while the running maximum lies within +-kStWindow; when it
// does not, the reference follows the running maximum (integer, at most 2
// below it), so that the dominant terms never carry the rounding of a large
// z.  needs_move says whether the running maximum rr (relative to ref) breaks
// the rule.
__device__ __forceinline__ bool needs_move(float rr, float ref) {
  return ref == 0.f ? !(fabsf(rr) <= kStWindow) : !(rr <= 2.f && rr >= -kStWindow);
}

// Apply the rule: new reference, exact power-of-two rescaling of the sum.
__device__ __forceinline__ void move_ref(float& rr, float& ref, float& S) {
  if (!(rr > -INFINITY) || !needs_move(rr, ref)) return;   // no terms yet, or nothing to do
  const float ymax = rr + ref;
  const float nr = fabsf(ymax) <= kStWindow ? 0.f : rintf(ymax);
  S = scale2(S, ref - nr);
  rr = ymax - nr;
  ref = nr;
}


// Buffers of one half-step (as in the striped passes): a trial column pass
// reads f' and is shifted by h = f_k^{C,eps}.
struct PassIo {
  int mode, cf, sh_g, dst_g;
  Split red, outs;
};

__device__ __forceinline__ PassIo pass_io(const Prob& P, bool col, int mode, int cf, int cg) {
  PassIo io;
  io.mode = mode;
  io.cf = cf;
  int src_f = cf;
  io.sh_g = cg;
  io.dst_g = (cg + 1) % 3;
  if (col && mode == MODE_TRIAL) {
    src_f = 1 - cf;
    io.sh_g = (cg + 1) % 3;
    io.dst_g = (cg + 2) % 3;
  }
  if (mode == MODE_EVAL) io.dst_g = -1;
  io.red = col ? P.rs[src_f] : P.cs[cg];
  io.outs = col ? P.cs[io.sh_g] : P.rs[cf];
  return io;
}

}  // namespace eotk
