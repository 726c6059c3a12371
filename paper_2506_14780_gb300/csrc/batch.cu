// Persistent batched log-domain Sinkhorn (eot_solve_batch): many problems of
// uneven size and eps run the iteration of the single solves -- Sinkhorn
// half-steps (Eq. foc_f, Eq. foc_g; Eq. SK_iterations), the L1 marginal test
// of Algorithm 4.1 at the pair (f_k, g_k), eps continuation (Sec. 5), the
// exact exponent split of eot_device.cuh and the final verification of the
// float32 estimate -- inside ONE cooperative launch.
//
// Scheduling.  A problem is a task run by a gang of G CTAs (G a power of two
// picked per problem by the host from a cost model that it calibrates once per
// device on synthetic problems: element rate, fixed cost of an iteration, cost
// of a gang barrier).  The host lists the tasks longest predicted first, each
// task G times (ranks
// 0..G-1); every CTA of the persistent grid takes the next entry of that list
// with an atomic counter, so a gang forms from the first CTAs that free up.
// Entries are taken in order and every task ends (iteration caps and bounded
// waits), so with all CTAs resident (cooperative launch) only the gang being
// formed can wait, and it completes as CTAs finish earlier tasks.
//
// Within a task the gang splits the rows (row half-step) and the columns
// (column half-step) into contiguous ranges: every output potential is
// computed whole by one CTA, so no partial log-sum-exp states cross CTAs, and
// the order of every sum depends on the problem's shape alone.  Gang barriers
// (global counters, acquire/release, time-bounded waits) separate the
// half-steps; the L1 test and the scores are summed by every rank over the
// whole problem in one fixed order, so a result does not depend on the gang
// size, on the schedule or on the other problems of the batch.
// The column half-step writes the new g into the other of two buffers and the
// gang commits it only when the test fails, so that the returned pair is
// (f_k, g_k) of the stopping iteration (as in the single solves).
//
// Inner loops: the cost is read with 16-byte loads, eight per lane issued
// before the arithmetic (enough bytes in flight per SM to stream from HBM);
// exponents are formed two at a time with the packed float32x2 instructions;
// the float64 finish of each output (log, delta update, grid splits) runs in
// whole warps, batched per chunk of rows or columns.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "eot_device.cuh"
#include "eot_internal.h"
#include "stream_common.cuh"
#include "batch.h"

namespace eotk {

__device__ __forceinline__ unsigned long long gtime_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_rel(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier of the G CTAs of a gang (G == 1: the CTA barrier).  Returns false
// (in every thread) if the wait exceeded wait_ns and gave up.
__device__ bool gang_sync(unsigned* bar, int G, unsigned long long wait_ns, int* s_flag) {
  __syncthreads();
  if (G > 1 && threadIdx.x == 0) {
    bool ok = true;
    const unsigned gen = ld_acq(&bar[1]);
    if (arrive_count(&bar[0]) == (unsigned)(G - 1)) {
      bar[0] = 0u;
      st_rel(&bar[1], gen + 1u);
    } else {
      const unsigned long long t0 = gtime_ns();
      while (ld_acq(&bar[1]) == gen) {
        if (gtime_ns() - t0 > wait_ns) {
          ok = false;
          break;
        }
        __nanosleep(64);
      }
    }
    *s_flag = ok ? 0 : 1;
  } else if (threadIdx.x == 0) {
    *s_flag = 0;
  }
  __syncthreads();
  return *s_flag == 0;
}

// Split of a potential value into the four exponent arrays (eot_device.cuh);
// the low parts are stored times k2 = 1/(eps ln 2) of the current level, so
// that an exponent needs no further product for them.
__device__ __forceinline__ void bsplit(const BatchTask& T, double o, double eps_logw, float k2,
                                       Split s, int idx) {
  double hi;
  float lo;
  split_grid(o + eps_logw, T.qscale, T.qinv, hi, lo);
  s.A[idx] = (float)(hi + (double)T.M);
  s.AL[idx] = lo * k2;
  split_grid(o, T.qscale, T.qinv, hi, lo);
  s.K[idx] = (float)((double)T.M - hi);
  s.KL[idx] = lo * k2;
}

// Finish one output index from its merged state (reference R and sum S in
// log2 units, without the output side's low part kl, which enters here): the
// new value (delta form: out = shift - eps L, Eq. foc_f / foc_g), its splits
// (unless eval) and L.  A non-finite or out-of-range value raises the
// problem's numeric flag and keeps the old value.
__device__ __forceinline__ void bfinish(const BatchTask& T, float R, float S, float kl,
                                        double shift, double eps_logw, double eps, float k2,
                                        double* out, Split so, float* Lout, int idx, bool eval) {
  double L = ((double)R + (double)kl) * 0.6931471805599453 + (double)log_sum((double)S);
  double o = shift - eps * L;
  if (!isfinite(o) || !(S > 0.f) || fabs(o) > T.pot_bound) {
    atomicOr(T.flag, 1u);
    o = shift;
    L = 0.0;
  }
  Lout[idx] = (float)L;
  if (!eval) {
    out[idx] = o;
    bsplit(T, o, eps_logw, k2, so, idx);
  }
}

// Rescale a pair of partial sums that share one reference.
__device__ __forceinline__ void move_ref2(float& rr, float& ref, float2& S) {
  const float old = ref;
  move_ref(rr, ref, S.x);
  if (ref != old) S.y = scale2(S.y, old - ref);
}

struct BShared {
  float4 cref[2][8][32];   // column pass: [buffer][row group][lane], 4 columns a lane
  float4 csum[2][8][32];
  float rref[2][256];      // row pass: [buffer][row of the chunk]
  float rsum[2][256];
  double red[8][8];        // block sums: [value][warp]
  int flag;
  int slot;
};

// Sum over the CTA of NV values per thread in a fixed order (warp butterflies,
// then the warps in index order); every thread receives the sums.
template <int NV, class V>
__device__ __forceinline__ void bsum_all(V v[NV], BShared& sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0) sh.red[k][wid] = (double)v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    V t = V(0);
    for (int w = 0; w < kBThreads / 32; ++w) t += (V)sh.red[k][w];
    v[k] = t;
  }
  __syncthreads();
}

// Partial log-sum-exp of row i over one lane's 4-column groups g = sub,
// sub + LPR, ... (eight groups per step, all cost loads issued first):
// exponents y_j = t (k2 + k2lo) + AL_j k2 in log2 units with the exact
// t = (A_j - K_i) - C_ij (k2lo: the float32 remainder of 1/(eps ln 2), so
// that the iteration is at eps itself), summed in a pair of float32 sums
// under one windowed reference.
template <bool ACC>
__device__ __forceinline__ void brow_stream(const BatchTask& T, const Split& cs, int i, int sub,
                                            int LPR, float k2, float k2lo, float& rf, float& ss) {
  const int m = T.m, ng = (m + 3) >> 2;
  const float4* Ci = reinterpret_cast<const float4*>(T.C + (size_t)i * T.pitch);
  const float4* A4 = reinterpret_cast<const float4*>(cs.A);
  const float4* L4 = reinterpret_cast<const float4*>(cs.AL);
  const float Ki = T.fs.K[i];
  const float2 nk = f2(-Ki, -Ki), k2v = f2(k2, k2), k2l = f2(k2lo, k2lo), m1 = f2(-1.f, -1.f);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float ref = 0.f, rr = -INFINITY;
  float2 S = f2(0.f, 0.f);
  for (int g0 = sub; g0 < ng; g0 += kBRowU * LPR) {
    float4 c[kBRowU];
#pragma unroll
    for (int u = 0; u < kBRowU; ++u) {
      const int g = g0 + u * LPR;
      c[u] = g < ng ? __ldcg(Ci + g) : z4;
    }
#pragma unroll
    for (int u = 0; u < kBRowU; ++u) {   // the lane's next step into L2
      const int g = g0 + (kBRowU + u) * LPR;
      if (g < ng) asm volatile("prefetch.global.L2 [%0];" ::"l"(Ci + g));
    }
    // exponents: the iteration rounds y = t k2 + AL once; an evaluation pass
    // (ACC) keeps t and forms y as p + q at the term, p = t k2 rounded and q
    // its exact rounding error plus AL (ex2_pq)
    float2 ya[kBRowU], yb[kBRowU];
#pragma unroll
    for (int u = 0; u < kBRowU; ++u) {
      const int g = g0 + u * LPR;
      const float4 a = g < ng ? A4[g] : z4;
      const float4 l = g < ng ? L4[g] : z4;
      const float2 ta = __ffma2_rn(f2(c[u].x, c[u].y), m1, __fadd2_rn(f2(a.x, a.y), nk));
      const float2 tb = __ffma2_rn(f2(c[u].z, c[u].w), m1, __fadd2_rn(f2(a.z, a.w), nk));
      if constexpr (ACC) {
        ya[u] = ta;
        yb[u] = tb;
      } else {
        ya[u] = __ffma2_rn(ta, k2v, __ffma2_rn(ta, k2l, f2(l.x, l.y)));
        yb[u] = __ffma2_rn(tb, k2v, __ffma2_rn(tb, k2l, f2(l.z, l.w)));
      }
      const int j = 4 * g;
      if (j + 3 >= m) {   // the ragged last group, or past the end of the row
        ya[u].x = j + 0 < m ? ya[u].x : -INFINITY;
        ya[u].y = j + 1 < m ? ya[u].y : -INFINITY;
        yb[u].x = j + 2 < m ? yb[u].x : -INFINITY;
        yb[u].y = j + 3 < m ? yb[u].y : -INFINITY;
      }
    }
    // the running maximum from the raw exponents (subtracting the reference
    // is monotone, so max(y) - ref = max(y - ref) exactly), then the terms
    float my = -INFINITY;
#pragma unroll
    for (int u = 0; u < kBRowU; ++u) {
      if constexpr (ACC) {
        const float2 pa = __fmul2_rn(ya[u], k2v), pb = __fmul2_rn(yb[u], k2v);
        my = fmaxf(my, fmaxf(fmaxf(pa.x, pa.y), fmaxf(pb.x, pb.y)));
      } else {
        my = fmaxf(my, fmaxf(fmaxf(ya[u].x, ya[u].y), fmaxf(yb[u].x, yb[u].y)));
      }
    }
    rr = fmaxf(rr, ref == 0.f ? my : my - ref);
    if (rr > -INFINITY && needs_move(rr, ref)) move_ref2(rr, ref, S);
    const bool r0 = ref == 0.f;
    const float2 nr = f2(-ref, -ref);
    if constexpr (ACC) {
      // evaluation: terms 2^(p + q) added one group after another (few live
      // registers; the order is fixed by the row's layout)
      float2 e = f2(0.f, 0.f);
#pragma unroll 2
      for (int u = 0; u < kBRowU; ++u) {
        const int g = g0 + u * LPR;
        const float4 l = g < ng ? L4[g] : z4;
        const float2 pa = __fmul2_rn(ya[u], k2v), pb = __fmul2_rn(yb[u], k2v);
        const float2 qa = __fadd2_rn(__ffma2_rn(ya[u], k2v, f2(-pa.x, -pa.y)),
                                     __ffma2_rn(ya[u], k2l, f2(l.x, l.y)));
        const float2 qb = __fadd2_rn(__ffma2_rn(yb[u], k2v, f2(-pb.x, -pb.y)),
                                     __ffma2_rn(yb[u], k2l, f2(l.z, l.w)));
        e = __fadd2_rn(e, f2(ex2_pq(__fsub_rn(pa.x, ref), qa.x) + ex2_pq(__fsub_rn(pb.x, ref), qb.x),
                             ex2_pq(__fsub_rn(pa.y, ref), qa.y) + ex2_pq(__fsub_rn(pb.y, ref), qb.y)));
      }
      S = __fadd2_rn(S, e);
    } else {
      float2 e[kBRowU];
#pragma unroll
      for (int u = 0; u < kBRowU; ++u)
        e[u] = r0 ? __fadd2_rn(ex2_2(ya[u]), ex2_2(yb[u]))
                  : __fadd2_rn(ex2_2(__fadd2_rn(ya[u], nr)), ex2_2(__fadd2_rn(yb[u], nr)));
#pragma unroll
      for (int w = 1; w < kBRowU; w *= 2)
#pragma unroll
        for (int u = 0; u + w < kBRowU; u += 2 * w) e[u] = __fadd2_rn(e[u], e[u + w]);
      S = __fadd2_rn(S, e[0]);
    }
  }
  ss = S.x + S.y;
  rf = ref;
}

// Row half-step over rows [r0, r1): f_i <- f_i - eps L_i (Eq. foc_f, delta
// form), g from buffer gi; eval: L only.  A row is reduced by a group of LPR
// lanes (a function of m alone, so every row sums in the same order whatever
// the gang or the tile); the rows go in chunks of at least RPW rows a warp
// (the task's tile), whose states pass through shared memory to warp 0, which
// finishes a whole chunk with full warps (the finish is float64 work, slow on
// this GPU) while the other warps stream the next chunk.
template <int RPW>
__device__ __forceinline__ void brow_pass(const BatchTask& T, int r0, int r1, int gi, double eps,
                                       float k2, float k2lo, bool eval, BShared& sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int LPR = T.lpr, rpw = 32 / LPR, sub = lane & (LPR - 1), grp = lane / LPR;
  const int rpwc = max(rpw, RPW), CR = (kBThreads / 32) * rpwc;
  const Split cs = T.gsp[gi];
  int k = 0;
  for (int q0 = r0; q0 < r1; q0 += CR, ++k) {
    const int buf = k & 1;
    for (int s = 0; s < rpwc; s += rpw) {
      const int lr = wid * rpwc + s + grp;
      const int i = q0 + lr;
      float rf = 0.f, ss = 0.f;
      if (i < r1) {
        if (eval) brow_stream<true>(T, cs, i, sub, LPR, k2, k2lo, rf, ss);
        else brow_stream<false>(T, cs, i, sub, LPR, k2, k2lo, rf, ss);
      }
      for (int o = LPR >> 1; o > 0; o >>= 1) {
        const float r2 = __shfl_xor_sync(0xffffffffu, rf, o);
        const float s2 = __shfl_xor_sync(0xffffffffu, ss, o);
        lse2_merge(rf, ss, r2, s2);
      }
      if (sub == 0 && EOT_CHECK(lr < 256, 602)) {
        sh.rref[buf][lr] = rf;
        sh.rsum[buf][lr] = ss;
      }
    }
    __syncthreads();
    if (wid == 0) {
      for (int lr = lane; lr < CR; lr += 32) {
        const int i = q0 + lr;
        if (i < r1)
          bfinish(T, sh.rref[buf][lr], sh.rsum[buf][lr], T.fs.KL[i], T.f[i], eps * T.loga[i], eps,
                  k2, T.f, T.fs, T.Lrow, i, eval);
      }
    }
  }
}

// Partial log-sum-exp of the CPL columns j..j+CPL-1 (CPL = 4 or 2: the
// column tile of the task, 32 CPL columns a block) over the 8-row blocks
// b = rg, rg + 8, ... (rg: the warp's row group): exponents
// t (k2 + k2lo) + AL_i k2 with the exact t = (A_i - K_j) - C_ij, windowed
// references per column and compensated pair sums (one compensated add per
// block of eight rows).  Every column's arithmetic is its own (a reference
// move folds the carried error of the moved column only), so a column's sum
// does not depend on CPL: the tile is a pure schedule choice.
template <bool ACC, int CPL>
__device__ __forceinline__ void bcol_stream(const BatchTask& T, const Split& os, int j, int c1,
                                            int rg, float k2, float k2lo, float (&Rout)[CPL],
                                            float (&Sout)[CPL]) {
  static_assert(CPL == 2 || CPL == 4, "2 or 4 columns a lane");
  constexpr int NP = CPL / 2;   // float2 pairs of columns
  const int n = T.n;
  const size_t pitch = (size_t)T.pitch;
  float2 nK[NP];
  if constexpr (CPL == 4) {
    const float4 K = *reinterpret_cast<const float4*>(os.K + j);
    nK[0] = f2(-K.x, -K.y);
    nK[1] = f2(-K.z, -K.w);
  } else {
    const float2 K = *reinterpret_cast<const float2*>(os.K + j);
    nK[0] = f2(-K.x, -K.y);
  }
  const float2 k2v = f2(k2, k2), k2l = f2(k2lo, k2lo), m1 = f2(-1.f, -1.f);
  const bool fullc = j + CPL <= c1;
  const float* Cj = T.C + j;
  float ref[CPL], rr[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) {
    ref[q] = 0.f;
    rr[q] = -INFINITY;
  }
  bool ref0 = true;
  float2 Sa[NP], Ca[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    Sa[p] = f2(0.f, 0.f);
    Ca[p] = f2(0.f, 0.f);
  }
  for (int b = rg; 8 * b < n; b += kBThreads / 32) {
    const int i0 = 8 * b;
    const bool fullr = i0 + 8 <= n;
    float2 c[8][NP];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = fullr || i0 + u < n;
      const float* src = Cj + (size_t)(i0 + u) * pitch;
      if constexpr (CPL == 4) {
        const float4 v = in ? __ldcg(reinterpret_cast<const float4*>(src))
                            : make_float4(0.f, 0.f, 0.f, 0.f);
        c[u][0] = f2(v.x, v.y);
        c[u][1] = f2(v.z, v.w);
      } else {
        c[u][0] = in ? __ldcg(reinterpret_cast<const float2*>(src)) : f2(0.f, 0.f);
      }
    }
    // the warp's next block into L2 while this one is reduced (measured on
    // the mixed 512-problem batch, with the row pass's prefetch: 0.45 -> 0.42 s)
    {
      const int in = i0 + 8 * (kBThreads / 32);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (in + u < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(Cj + (size_t)(in + u) * pitch));
    }
    const float4 a0 = *reinterpret_cast<const float4*>(T.fs.A + i0);
    const float4 a1 = *reinterpret_cast<const float4*>(T.fs.A + i0 + 4);
    const float4 l0 = *reinterpret_cast<const float4*>(T.fs.AL + i0);
    const float4 l1 = *reinterpret_cast<const float4*>(T.fs.AL + i0 + 4);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float lv[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
    // exponents as in the row pass: rounded once, or t kept for ACC
    float2 y[8][NP];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float2 arr = f2(av[u], av[u]), alr = f2(lv[u], lv[u]);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float2 t = __ffma2_rn(c[u][p], m1, __fadd2_rn(arr, nK[p]));
        if constexpr (ACC) y[u][p] = t;
        else y[u][p] = __ffma2_rn(t, k2v, __ffma2_rn(t, k2l, alr));
      }
    }
    if (!(fullr && fullc)) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool rv = i0 + u < n;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          y[u][p].x = (rv && j + 2 * p < c1) ? y[u][p].x : -INFINITY;
          y[u][p].y = (rv && j + 2 * p + 1 < c1) ? y[u][p].y : -INFINITY;
        }
      }
    }
    // running maxima from the raw exponents (max(y) - ref = max(y - ref))
    float my[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) my[q] = -INFINITY;
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        float2 pv = y[u][p];
        if constexpr (ACC) pv = __fmul2_rn(pv, k2v);
        my[2 * p] = fmaxf(my[2 * p], pv.x);
        my[2 * p + 1] = fmaxf(my[2 * p + 1], pv.y);
      }
    bool mv[CPL];
    bool move = false;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      rr[q] = fmaxf(rr[q], ref0 ? my[q] : my[q] - ref[q]);
      mv[q] = rr[q] > -INFINITY && needs_move(rr[q], ref[q]);
      move |= mv[q];
    }
    if (move) {
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if (mv[2 * p]) {
          Sa[p].x = __fmaf_rn(Ca[p].x, -1.f, Sa[p].x);
          Ca[p].x = 0.f;
          move_ref(rr[2 * p], ref[2 * p], Sa[p].x);
        }
        if (mv[2 * p + 1]) {
          Sa[p].y = __fmaf_rn(Ca[p].y, -1.f, Sa[p].y);
          Ca[p].y = 0.f;
          move_ref(rr[2 * p + 1], ref[2 * p + 1], Sa[p].y);
        }
      }
      ref0 = true;
#pragma unroll
      for (int q = 0; q < CPL; ++q) ref0 = ref0 && ref[q] == 0.f;
    }
    float2 nr[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) nr[p] = f2(-ref[2 * p], -ref[2 * p + 1]);
    if constexpr (ACC) {
      // evaluation: terms 2^(p + q), one row after another
      float2 e[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p) e[p] = f2(0.f, 0.f);
#pragma unroll 2
      for (int u = 0; u < 8; ++u) {
        const float2 alr = f2(lv[u], lv[u]);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float2 pp = __fmul2_rn(y[u][p], k2v);
          const float2 qq = __fadd2_rn(__ffma2_rn(y[u][p], k2v, f2(-pp.x, -pp.y)),
                                       __ffma2_rn(y[u][p], k2l, alr));
          e[p] = __fadd2_rn(e[p], f2(ex2_pq(__fsub_rn(pp.x, ref[2 * p]), qq.x),
                                     ex2_pq(__fsub_rn(pp.y, ref[2 * p + 1]), qq.y)));
        }
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) kahan_add2(Sa[p], Ca[p], e[p]);
    } else {
      float2 e[8][NP];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int p = 0; p < NP; ++p) e[u][p] = ex2_2(ref0 ? y[u][p] : __fadd2_rn(y[u][p], nr[p]));
#pragma unroll
      for (int w = 1; w < 8; w *= 2)
#pragma unroll
        for (int u = 0; u + w < 8; u += 2 * w)
#pragma unroll
          for (int p = 0; p < NP; ++p) e[u][p] = __fadd2_rn(e[u][p], e[u + w][p]);
#pragma unroll
      for (int p = 0; p < NP; ++p) kahan_add2(Sa[p], Ca[p], e[0][p]);
    }
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    kahan_fold2(Sa[p], Ca[p]);
    Rout[2 * p] = ref[2 * p];
    Rout[2 * p + 1] = ref[2 * p + 1];
    Sout[2 * p] = Sa[p].x;
    Sout[2 * p + 1] = Sa[p].y;
  }
}

__device__ __forceinline__ void lse_merge4(float4& R, float4& S, float4 r, float4 s) {
  lse2_merge(R.x, S.x, r.x, s.x);
  lse2_merge(R.y, S.y, r.y, s.y);
  lse2_merge(R.z, S.z, r.z, s.z);
  lse2_merge(R.w, S.w, r.w, s.w);
}

// Column half-step over columns [c0, c1) (c0 a multiple of 4): g'_j = g_j -
// eps L_j (Eq. foc_g, delta form) from buffer gi into buffer 1 - gi.  Blocks
// of 32 CPL columns, CPL a lane; each warp is one of eight row groups (8-row
// blocks, interleaved), whose states warp 0 merges in group order and
// finishes while the others stream the next block.  The order of every sum
// depends on n alone, not on the gang or on CPL.
template <int CPL>
__device__ __forceinline__ void bcol_pass(const BatchTask& T, int c0, int c1, int gi, double eps,
                                       float k2, float k2lo, bool eval, BShared& sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const Split os = T.gsp[gi];
  const Split ns = T.gsp[1 - gi];
  const double* gcur = T.g[gi];
  double* gnew = T.g[1 - gi];
  int k = 0;
  for (int cb = c0; cb < c1; cb += 32 * CPL, ++k) {
    const int buf = k & 1;
    const int j = cb + CPL * lane;
    float R[CPL], S[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) R[q] = S[q] = 0.f;
    if (j < c1) {
      if (eval) bcol_stream<true, CPL>(T, os, j, c1, wid, k2, k2lo, R, S);
      else bcol_stream<false, CPL>(T, os, j, c1, wid, k2, k2lo, R, S);
    }
    sh.cref[buf][wid][lane] = make_float4(R[0], R[1], CPL == 4 ? R[CPL - 2] : 0.f,
                                          CPL == 4 ? R[CPL - 1] : 0.f);
    sh.csum[buf][wid][lane] = make_float4(S[0], S[1], CPL == 4 ? S[CPL - 2] : 0.f,
                                          CPL == 4 ? S[CPL - 1] : 0.f);
    __syncthreads();
    if (wid == 0 && j < c1) {
      float4 R4 = sh.cref[buf][0][lane], S4 = sh.csum[buf][0][lane];
      for (int g2 = 1; g2 < kBThreads / 32; ++g2)
        lse_merge4(R4, S4, sh.cref[buf][g2][lane], sh.csum[buf][g2][lane]);
      const float rv[4] = {R4.x, R4.y, R4.z, R4.w}, sv[4] = {S4.x, S4.y, S4.z, S4.w};
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const int jj = j + q;
        if (jj < c1)
          bfinish(T, rv[q], sv[q], os.KL[jj], gcur[jj], eps * T.logb[jj], eps, k2, gnew, ns,
                  T.Lcol, jj, eval);
      }
    }
  }
}

// The task's tile (BatchTask::tile, a template argument of brun_task): bit 0,
// two columns a lane in the column half-step (64-column blocks) instead of
// four; bit 1, at least eight rows a warp per chunk of the row half-step
// instead of four.
template <int TILE>
__device__ __forceinline__ void bcol_pass_t(const BatchTask& T, int c0, int c1, int gi, double eps,
                                            float k2, float k2lo, bool eval, BShared& sh) {
  bcol_pass<(TILE & 1) ? 2 : 4>(T, c0, c1, gi, eps, k2, k2lo, eval, sh);
}
template <int TILE>
__device__ __forceinline__ void brow_pass_t(const BatchTask& T, int r0, int r1, int gi, double eps,
                                            float k2, float k2lo, bool eval, BShared& sh) {
  brow_pass<(TILE & 2) ? 8 : 4>(T, r0, r1, gi, eps, k2, k2lo, eval, sh);
}

// One task (problem) run by rank `rank` of its gang.  Gang-wide sums (the L1
// test, the scores) are formed by every rank from the per-index arrays in one
// fixed order, so they, and with them every decision, do not depend on G.
template <int TILE>
__device__ void brun_task(const BatchTask& T, int rank, BShared& sh) {
  const int G = T.G, n = T.n, m = T.m;
  const int r0 = (int)((long long)n * rank / G), r1 = (int)((long long)n * (rank + 1) / G);
  const int nq = (m + 3) >> 2;
  const int c0 = 4 * (int)((long long)nq * rank / G);
  const int c1 = min(m, 4 * (int)((long long)nq * (rank + 1) / G));
  int gi = 0, total = 0, iter = 0, status = 0, verify_rounds = 0, lev = 0;
  double row_l1 = 0.0, col_l1 = 0.0;
  bool have_row = false;
  const unsigned long long t_begin = gtime_ns();
  unsigned long long t_last = t_begin;
  auto sync = [&]() -> bool {
    if (gang_sync(T.bar, G, T.wait_ns, &sh.flag)) return true;
    status = 4;
    return false;
  };
  auto numeric = [&]() { return *(volatile const unsigned*)T.flag != 0u; };
  // sum_k w_k |expm1 L_k| over a whole side, in float (the test needs a few digits)
  auto l1_side = [&](const float* L, const float* w, int len) -> double {
    float v[1] = {0.f};
    for (int k = threadIdx.x; k < len; k += kBThreads) v[0] += w[k] * fabsf(expm1f(L[k]));
    bsum_all<1>(v, sh);
    return (double)v[0];
  };
  for (lev = 0; lev < T.nlev && status == 0; ++lev) {
    const bool last = lev == T.nlev - 1;
    const double eps = T.eps[lev];
    const double k2d = 1.0 / (eps * 0.6931471805599453);
    const float k2 = (float)k2d, k2lo = (float)(k2d - (double)k2);
    if (last) t_last = gtime_ns();
    // splits of the carried potentials at this eps
    for (int i = r0 + threadIdx.x; i < r1; i += kBThreads) bsplit(T, T.f[i], eps * T.loga[i], k2, T.fs, i);
    for (int j = c0 + threadIdx.x; j < c1; j += kBThreads)
      bsplit(T, T.g[gi][j], eps * T.logb[j], k2, T.gsp[gi], j);
    if (!sync()) break;
    // g_1 = f_0^{C,eps} (Algorithm 4.1 line 3 at the first iteration)
    bcol_pass_t<TILE>(T, c0, c1, gi, eps, k2, k2lo, false, sh);
    if (!sync()) break;
    if (numeric()) {
      status = 3;
      break;
    }
    gi ^= 1;
    double tol = last ? T.tol_last : T.tol_level;
    iter = 0;
    // the stall check of stop_code, in local state (every CTA of the gang
    // computes the same l1 and takes the same decision)
    double stall_l1 = 1e300;
    int stall_at = T.stall_window;
    for (;;) {
      brow_pass_t<TILE>(T, r0, r1, gi, eps, k2, k2lo, false, sh);   // f_k = g_k^{C,eps}
      if (!sync()) break;
      bcol_pass_t<TILE>(T, c0, c1, gi, eps, k2, k2lo, false, sh);   // f_k^{C,eps}: the L1 test
      if (!sync()) break;
      const double l1 = l1_side(T.Lcol, T.bf, m);
      ++iter;
      ++total;
      if (numeric()) {
        status = 3;
        break;
      }
      col_l1 = l1;
      if (l1 < tol) {
        if (!last) break;
        // verify the pair (f_k, g_k): both terms of the L1 error with the
        // unbiased exponential (the two passes read f_k, g_k and write
        // different arrays: one barrier after both)
        brow_pass_t<TILE>(T, r0, r1, gi, eps, k2, k2lo, true, sh);
        bcol_pass_t<TILE>(T, c0, c1, gi, eps, k2, k2lo, true, sh);
        if (!sync()) break;
        row_l1 = l1_side(T.Lrow, T.af, n);
        col_l1 = l1_side(T.Lcol, T.bf, m);
        have_row = true;
        ++verify_rounds;
        if (row_l1 + col_l1 < T.tol_verify || verify_rounds >= 4) break;
        // continue with the fast test's threshold scaled to what the
        // verification found
        tol = 0.9 * (T.tol_verify - row_l1) * (l1 / fmax(col_l1, 1e-300));
        if (!(tol > 0.0) || tol > l1) tol = 0.5 * l1;
        have_row = false;
        continue;
      }
      if (iter >= T.max_iter) {
        status = 2;
        break;
      }
      if (T.stall_window > 0 && iter >= stall_at) {
        const bool stalled = !(l1 < 0.99 * stall_l1);
        stall_l1 = l1;
        stall_at = iter + T.stall_window;
        if (stalled) {   // an intermediate level goes on to the next eps
          if (last) status = 6;
          break;
        }
      }
      gi ^= 1;   // commit g_{k+1} = f_k^{C,eps}
    }
  }
  const int levels = lev;
  if (status == 0) status = 1;
  if (status != 4) {
    // scores of the returned pair (f, g[gi]) at the last eps, from the
    // log-ratios of the verification passes (unbiased exponential)
    const double eps = T.eps[max(0, min(levels, T.nlev) - 1)];
    const double k2d = 1.0 / (eps * 0.6931471805599453);
    const float k2 = (float)k2d, k2lo = (float)(k2d - (double)k2);
    bool ok = true;
    if (!have_row) {
      brow_pass_t<TILE>(T, r0, r1, gi, eps, k2, k2lo, true, sh);
      bcol_pass_t<TILE>(T, c0, c1, gi, eps, k2, k2lo, true, sh);
      ok = sync();
      if (ok) row_l1 = l1_side(T.Lrow, T.af, n);
    }
    if (ok) {
      // float64 sums, whole problem, fixed order: <f,a>, sum pi, <pi1-a,f>,
      // <g,b>, <pi^T1-b,g>, column L1, <h,b> with h = f^{C,eps} from the
      // last column half-step (the other buffer)
      double v[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int i = threadIdx.x; i < n; i += kBThreads) {
        const double e = (double)expm1f(T.Lrow[i]), ai = T.a[i], fi = T.f[i];
        v[0] += ai * fi;
        v[1] += ai * (1.0 + e);
        v[2] += ai * e * fi;
      }
      const double *gc = T.g[gi], *gh = T.g[1 - gi];
      for (int j = threadIdx.x; j < m; j += kBThreads) {
        const double e = (double)expm1f(T.Lcol[j]), bj = T.b[j], gj = gc[j];
        v[3] += bj * gj;
        v[4] += bj * e * gj;
        v[5] += bj * fabs(e);
        v[6] += bj * gh[j];
      }
      bsum_all<7>(v, sh);
      const double fa = v[0], sumpi = v[1], gap_f = v[2];
      const double gb = v[3], gap_g = v[4], cl1 = v[5], sum_bh = v[6];
      const double c = 0.5 * (gb - fa);
      for (int i = r0 + threadIdx.x; i < r1; i += kBThreads) T.f_out[i] = T.f[i] + c;
      for (int j = c0 + threadIdx.x; j < c1; j += kBThreads) T.g_out[j] = gc[j] - c;
      if (rank == 0 && threadIdx.x == 0) {
        BatchOut* o = T.out;
        o->row_l1 = row_l1;
        o->col_l1 = cl1;
        o->q_dual = fa + gb - eps * (sumpi - 1.0);
        o->q_semi = fa + sum_bh;
        o->dual_gap = gap_f + gap_g + eps * (sumpi - 1.0);
        o->gauge = c;
      }
    } else {
      status = 4;
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    BatchOut* o = T.out;
    o->status = status;
    o->iters = iter;
    o->total_iters = total;
    o->levels = levels;
    o->verify_rounds = verify_rounds;
    o->t_begin = t_begin;
    o->t_end = gtime_ns();
    o->t_last_level = t_last;
  }
}

__global__ void __launch_bounds__(kBThreads, 2) batch_sk_kernel(const BatchTask* __restrict__ tasks,
                                                              const int2* __restrict__ slots,
                                                              int nslots, unsigned* next_slot) {
  __shared__ BShared sh;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) sh.slot = (int)atomicAdd(next_slot, 1u);
    __syncthreads();
    const int s = sh.slot;
    if (s >= nslots) return;
    const int2 e = slots[s];
    const BatchTask& T = tasks[e.x];
    if (!EOT_CHECK(e.y >= 0 && e.y < T.G && T.G <= kBMaxGang, 601)) continue;
    switch (T.tile) {
      case 1: brun_task<1>(T, e.y, sh); break;
      case 2: brun_task<2>(T, e.y, sh); break;
      case 3: brun_task<3>(T, e.y, sh); break;
      default: brun_task<0>(T, e.y, sh); break;
    }
  }
}

// ---------------------------------------------------------------------------
// Set-up kernels over all problems of a batch.
// ---------------------------------------------------------------------------
// One CTA per (problem, side): w <- w / sum(w), log w; flags bad weights.
__global__ void __launch_bounds__(256) batch_weights_kernel(const BatchIn* __restrict__ in) {
  const BatchIn& P = in[blockIdx.x >> 1];
  const bool side_b = blockIdx.x & 1;
  const int len = side_b ? P.m : P.n;
  const double* win = side_b ? P.win_b : P.win_a;
  double* w = side_b ? P.b : P.a;
  double* lw = side_b ? P.logb : P.loga;
  float* wf = side_b ? P.bf : P.af;
  __shared__ double sh[8];
  double s = 0.0;
  unsigned nb = 0;
  for (int i = threadIdx.x; i < len; i += 256) {
    const double v = win[i];
    if (!(v > 0.0) || !isfinite(v)) ++nb;
    s += v;
  }
  s = warp_sum_d(s);
  for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, o);
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = s;
    if (nb) atomicAdd(&P.bad[0], nb);
  }
  __syncthreads();
  double tot = 0.0;
  for (int k = 0; k < 8; ++k) tot += sh[k];
  for (int i = threadIdx.x; i < len; i += 256) {
    const double v = win[i] / tot;
    w[i] = v;
    wf[i] = (float)v;
    lw[i] = v > 0.0 ? log(v) : -INFINITY;
  }
}

__device__ __forceinline__ double bsqdist(const float* __restrict__ x, const float* __restrict__ y,
                                          int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    const double t = __dsub_rn((double)x[k], (double)y[k]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}

// Pass 1: max of the cost (points: max ||x - y||^2 in float64; given C: max
// |C| and the non-finite count).  Grid (row blocks, problems); one warp per
// row, lanes over columns.
__global__ void __launch_bounds__(256) batch_cost_max_kernel(const BatchIn* __restrict__ in) {
  const BatchIn& P = in[blockIdx.y];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double mx = 0.0;
  unsigned nb = 0;
  for (int i = blockIdx.x * 8 + wid; i < P.n; i += gridDim.x * 8) {
    for (int j = lane; j < P.m; j += 32) {
      if (P.givenC) {
        const float v = P.Cin[(size_t)i * P.m + j];
        if (!isfinite(v)) ++nb;
        else mx = fmax(mx, (double)fabsf(v));
      } else {
        mx = fmax(mx, bsqdist(P.X + (size_t)i * P.d, P.Y + (size_t)j * P.d, P.d));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  if (lane == 0) {
    atomicMax(P.cmax, (unsigned long long)__double_as_longlong(mx));
    if (nb) atomicAdd(&P.bad[1], nb);
  }
}

// Pass 2: C (pitched), rounded once to float32, optionally divided by the max
// (in float64, as the single solves).
__global__ void __launch_bounds__(256) batch_cost_fill_kernel(const BatchIn* __restrict__ in) {
  const BatchIn& P = in[blockIdx.y];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double cmax = __longlong_as_double((long long)*P.cmax);
  const bool norm = P.normalize && cmax > 0.0;
  for (int i = blockIdx.x * 8 + wid; i < P.n; i += gridDim.x * 8) {
    float* row = P.C + (size_t)i * P.pitch;
    for (int j = lane; j < P.pitch; j += 32) {
      float out = 0.f;
      if (j < P.m) {
        double v = P.givenC ? (double)P.Cin[P.trans ? (size_t)j * P.n + i : (size_t)i * P.m + j]
                            : bsqdist(P.X + (size_t)i * P.d, P.Y + (size_t)j * P.d, P.d);
        if (norm) v = __ddiv_rn(v, cmax);
        out = __double2float_rn(v);
      }
      row[j] = out;
    }
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
int batch_ctas_per_sm() {
  int k = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, batch_sk_kernel, kBThreads, 0);
  return k;
}

cudaError_t launch_batch_setup(const BatchIn* d_in, int count, int maxrows, cudaStream_t s) {
  batch_weights_kernel<<<2 * count, 256, 0, s>>>(d_in);
  const int bx = std::max(1, std::min((maxrows + 7) / 8, 64));
  batch_cost_max_kernel<<<dim3(bx, count), 256, 0, s>>>(d_in);
  batch_cost_fill_kernel<<<dim3(bx, count), 256, 0, s>>>(d_in);
  return cudaGetLastError();
}

cudaError_t launch_batch_sk(const BatchTask* d_tasks, const int2* d_slots, int nslots,
                            unsigned* d_next, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_sk_kernel, d_tasks, d_slots, nslots, d_next);
}

EOT_DEBUG_UNIT(batch)

}  // namespace eotk
