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
// computed whole by one CTA, so no partial log-sum-exp states cross CTAs.
// Gang barriers (global counters, acquire/release, time-bounded waits)
// separate the half-steps; per-rank partial sums, added in rank order, give
// the L1 test and the scores, so the results do not depend on scheduling.
// The column half-step writes the new g into the other of two buffers and the
// gang commits it only when the test fails, so that the returned pair is
// (f_k, g_k) of the stopping iteration (as in the single solves).
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
// (in every thread) if the wait gave up.
__device__ bool gang_sync(unsigned* bar, int G, int* s_flag) {
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
        if (gtime_ns() - t0 > kBWaitNs) {
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

// Running log-sum-exp of one output index over a thread's terms (log2 units,
// windowed integer reference as in the staged passes).
struct BLse {
  float ref, rr, S;
};

__device__ __forceinline__ void blse_add4(BLse& s, float y0, float y1, float y2, float y3) {
  float z0 = y0, z1 = y1, z2 = y2, z3 = y3;
  if (s.ref != 0.f) {
    z0 -= s.ref;
    z1 -= s.ref;
    z2 -= s.ref;
    z3 -= s.ref;
  }
  s.rr = fmaxf(s.rr, fmaxf(fmaxf(z0, z1), fmaxf(z2, z3)));
  if (s.rr > -INFINITY && needs_move(s.rr, s.ref)) {
    move_ref(s.rr, s.ref, s.S);
    z0 = y0 - s.ref;
    z1 = y1 - s.ref;
    z2 = y2 - s.ref;
    z3 = y3 - s.ref;
  }
  s.S += (ex2_approx(z0) + ex2_approx(z1)) + (ex2_approx(z2) + ex2_approx(z3));
}

// Split of a potential value into the four exponent arrays (eot_device.cuh).
__device__ __forceinline__ void bsplit(const BatchTask& T, double o, double eps_logw, Split s,
                                       int idx) {
  double hi;
  float lo;
  split_grid(o + eps_logw, T.qscale, T.qinv, hi, lo);
  s.A[idx] = (float)(hi + (double)T.M);
  s.AL[idx] = lo;
  split_grid(o, T.qscale, T.qinv, hi, lo);
  s.K[idx] = (float)((double)T.M - hi);
  s.KL[idx] = lo;
}

// Finish one output index from its merged (R, S) (log2 units): the new value
// (delta form: out = shift - eps L), its splits (unless eval), and, in float
// (the test needs a few digits of a sum of positive terms), its L1 term
// w |expm1 L| and a numeric flag.  Float64 work here is kept to the splits:
// it runs at a small fraction of the float32 rate on this GPU.
__device__ __forceinline__ void bfinish(const BatchTask& T, float R, float S, double shift,
                                        double w, double eps_logw, double eps, double* out,
                                        Split so, float* Lout, int idx, bool eval,
                                        float acc[2]) {
  float L = R * kLn2 + log_sum((double)S);
  double o = shift - eps * (double)L;
  if (!isfinite(o) || !(S > 0.f) || fabs(o) > T.pot_bound) {
    acc[1] += 1.f;
    o = shift;
    L = 0.f;
  }
  Lout[idx] = L;
  if (!eval) {
    out[idx] = o;
    bsplit(T, o, eps_logw, so, idx);
  }
  acc[0] += (float)w * fabsf(expm1f(L));
}

// Sum of two floats over the CTA; valid in thread 0.
__device__ __forceinline__ void bsum2f(float v[2], float* sh /*[2][8]*/) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float a = warp_sum_f(v[0]), b = warp_sum_f(v[1]);
  if (lane == 0) {
    sh[wid] = a;
    sh[8 + wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float x = 0.f, y = 0.f;
    for (int w = 0; w < kBThreads / 32; ++w) {
      x += sh[w];
      y += sh[8 + w];
    }
    v[0] = x;
    v[1] = y;
  }
  __syncthreads();
}

// Sum of four doubles over the CTA; valid in thread 0.
__device__ __forceinline__ void bsum4(double v[4], double* sh /*[4][8]*/) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double x = warp_sum_d(v[k]);
    if (lane == 0) sh[k * 8 + wid] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double t = 0.0;
      for (int w = 0; w < kBThreads / 32; ++w) t += sh[k * 8 + w];
      v[k] = t;
    }
  }
  __syncthreads();
}

struct BShared {
  float mr[kBThreads];
  float ms[kBThreads];
  double red[32];
  float redf[16];
  int flag;
  int slot;
};

// Row half-step over rows [r0, r1): f_i <- f_i - eps L_i (Eq. foc_f, delta
// form), g from buffer gi.  eval: log-ratios and sums only.  A row is reduced
// by a group of LPR lanes (a power of two sized so that a lane streams about
// four 4-column groups), so a warp finishes 32 / LPR rows at once.
__device__ void brow_pass(const BatchTask& T, int r0, int r1, int gi, double eps, float k2,
                          bool eval, float acc[2]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int m = T.m;
  const Split cs = T.gsp[gi];
  int LPR = 1;
  while (LPR < 32 && LPR * 16 < m) LPR *= 2;
  const int sub = lane & (LPR - 1), grp = lane / LPR, rpw = 32 / LPR;
  for (int i0 = r0 + wid * rpw; i0 < r1; i0 += (kBThreads / 32) * rpw) {
    const int i = i0 + grp;
    const bool iv = i < r1;
    float rf = -INFINITY, ss = 0.f;
    if (iv) {
      const float Ki = T.fs.K[i], cci = T.fs.KL[i] * k2;
      const float* Ci = T.C + (size_t)i * T.pitch;
      BLse s{0.f, -INFINITY, 0.f};
      // two 4-column groups per step, all loads issued before the arithmetic
      // (the cost rows are padded to a multiple of 4 floats and the split
      // arrays to a multiple of 128, so the 16-byte loads stay in bounds)
      auto terms = [&](int j, float4 c, float4 av, float4 al, float y[4]) {
        const float cv[4] = {c.x, c.y, c.z, c.w};
        const float aa[4] = {av.x, av.y, av.z, av.w};
        const float ll[4] = {al.x, al.y, al.z, al.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float t = __fsub_rn(__fsub_rn(aa[q], Ki), cv[q]);
          y[q] = (j + q < m) ? __fmaf_rn(t, k2, __fmaf_rn(ll[q], k2, cci)) : -INFINITY;
        }
      };
      const int step = LPR * 4;
      int j = sub * 4;
      for (; j + step < m; j += 2 * step) {
        const float4 c0 = *reinterpret_cast<const float4*>(Ci + j);
        const float4 c1 = *reinterpret_cast<const float4*>(Ci + j + step);
        const float4 a0 = __ldg(reinterpret_cast<const float4*>(cs.A + j));
        const float4 a1 = __ldg(reinterpret_cast<const float4*>(cs.A + j + step));
        const float4 l0 = __ldg(reinterpret_cast<const float4*>(cs.AL + j));
        const float4 l1 = __ldg(reinterpret_cast<const float4*>(cs.AL + j + step));
        float y0[4], y1[4];
        terms(j, c0, a0, l0, y0);
        terms(j + step, c1, a1, l1, y1);
        blse_add4(s, y0[0], y0[1], y0[2], y0[3]);
        blse_add4(s, y1[0], y1[1], y1[2], y1[3]);
      }
      if (j < m) {
        float y0[4];
        terms(j, *reinterpret_cast<const float4*>(Ci + j),
              __ldg(reinterpret_cast<const float4*>(cs.A + j)),
              __ldg(reinterpret_cast<const float4*>(cs.AL + j)), y0);
        blse_add4(s, y0[0], y0[1], y0[2], y0[3]);
      }
      rf = (s.S > 0.f) ? s.ref : -INFINITY;
      ss = s.S;
    }
    // merge the group's lanes (every lane of the warp takes part in the shuffles)
    for (int o = LPR >> 1; o > 0; o >>= 1) {
      const float r2 = __shfl_xor_sync(0xffffffffu, rf, o);
      const float s2 = __shfl_xor_sync(0xffffffffu, ss, o);
      lse2_merge(rf, ss, r2, s2);
    }
    if (iv && sub == 0)
      bfinish(T, rf, ss, T.f[i], T.a[i], eps * T.loga[i], eps, T.f, T.fs, T.Lrow, i, eval, acc);
  }
}

// Column half-step over columns [c0, c1): g'_j = g_j - eps L_j (Eq. foc_g,
// delta form) from buffer gi into buffer 1 - gi (unless eval).  Threads over
// columns (coalesced row segments); a range narrower than the CTA splits the
// rows among R groups whose states merge in shared memory.
__device__ void bcol_pass(const BatchTask& T, int c0, int c1, int gi, double eps, float k2,
                          bool eval, float acc[2], BShared& sh) {
  const int tid = threadIdx.x;
  const int n = T.n, w = c1 - c0;
  if (w <= 0) return;
  // W columns x R row groups: the fewest terms per thread (each block of W
  // columns adds a merge of R states), ties to the wider layout
  int W = 32;
  {
    long long best = -1;
    for (int Wc = 32; Wc <= kBThreads; Wc *= 2) {
      const int Rc = kBThreads / Wc;
      const long long blocks = (w + Wc - 1) / Wc;
      const long long cost = blocks * (((long long)n + Rc - 1) / Rc + 8 * Rc);
      if (best < 0 || cost <= best) {
        best = cost;
        W = Wc;
      }
    }
  }
  const int R = kBThreads / W;
  const int col = tid % W, rg = tid / W;
  const Split os = T.gsp[gi];
  const Split ns = T.gsp[1 - gi];
  const double* gcur = T.g[gi];
  double* gnew = T.g[1 - gi];
  for (int jb = c0; jb < c1; jb += W) {
    const int j = jb + col;
    const bool jv = j < c1 && rg < R;
    BLse s{0.f, -INFINITY, 0.f};
    if (jv) {
      const float Kj = os.K[j], ccj = os.KL[j] * k2;
      const float* Cj = T.C + j;
      int i = rg;
      // eight rows per step, all loads issued before the arithmetic
      for (; i + 7 * R < n; i += 8 * R) {
        float c[8], av[8], al[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int ii = i + u * R;
          c[u] = Cj[(size_t)ii * T.pitch];
          av[u] = __ldg(T.fs.A + ii);
          al[u] = __ldg(T.fs.AL + ii);
        }
        float y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float t = __fsub_rn(__fsub_rn(av[u], Kj), c[u]);
          y[u] = __fmaf_rn(t, k2, __fmaf_rn(al[u], k2, ccj));
        }
        blse_add4(s, y[0], y[1], y[2], y[3]);
        blse_add4(s, y[4], y[5], y[6], y[7]);
      }
      for (; i < n; i += R) {
        const float c = Cj[(size_t)i * T.pitch];
        const float t = __fsub_rn(__fsub_rn(__ldg(T.fs.A + i), Kj), c);
        const float y = __fmaf_rn(t, k2, __fmaf_rn(__ldg(T.fs.AL + i), k2, ccj));
        blse_add4(s, y, -INFINITY, -INFINITY, -INFINITY);
      }
    }
    sh.mr[tid] = (s.S > 0.f) ? s.ref : -INFINITY;
    sh.ms[tid] = s.S;
    __syncthreads();
    if (rg == 0 && jv) {
      float rf = sh.mr[col], ss = sh.ms[col];
      for (int g2 = 1; g2 < R; ++g2) lse2_merge(rf, ss, sh.mr[g2 * W + col], sh.ms[g2 * W + col]);
      bfinish(T, rf, ss, gcur[j], T.b[j], eps * T.logb[j], eps, gnew, ns, T.Lcol, j, eval, acc);
    }
    __syncthreads();
  }
}

// One task (problem) run by rank `rank` of its gang.
__device__ void brun_task(const BatchTask& T, int rank, BShared& sh) {
  const int G = T.G, n = T.n, m = T.m;
  const int r0 = (int)((long long)n * rank / G), r1 = (int)((long long)n * (rank + 1) / G);
  const int c0 = (int)((long long)m * rank / G), c1 = (int)((long long)m * (rank + 1) / G);
  double* my = T.part + (size_t)rank * kBPart;
  int gi = 0, total = 0, iter = 0, status = 0, verify_rounds = 0, lev = 0;
  double row_l1 = 0.0, col_l1 = 0.0;
  bool have_row = false;
  const unsigned long long t_begin = gtime_ns();
  unsigned long long t_last = t_begin;
  auto sync = [&]() -> bool {
    if (gang_sync(T.bar, G, &sh.flag)) return true;
    status = 4;
    return false;
  };
  // gang-wide sums of the partials (rank order)
  auto gsum = [&](int k) {
    double t = 0.0;
    for (int q = 0; q < G; ++q) t += __ldcg(T.part + (size_t)q * kBPart + k);
    return t;
  };
  auto publish = [&](double v[4], int base) {
    bsum4(v, sh.red);
    if (threadIdx.x == 0)
      for (int k = 0; k < 4; ++k) my[base + k] = v[k];
  };
  auto publishf = [&](float v[2], int base) {
    bsum2f(v, sh.redf);
    if (threadIdx.x == 0) {
      my[base] = (double)v[0];
      my[base + 1] = (double)v[1];
    }
  };
  for (lev = 0; lev < T.nlev && status == 0; ++lev) {
    const bool last = lev == T.nlev - 1;
    const double eps = T.eps[lev];
    const float k2 = (float)(1.0 / (eps * 0.6931471805599453));
    if (last) t_last = gtime_ns();
    // splits of the carried potentials at this eps
    for (int i = r0 + threadIdx.x; i < r1; i += kBThreads) bsplit(T, T.f[i], eps * T.loga[i], T.fs, i);
    for (int j = c0 + threadIdx.x; j < c1; j += kBThreads)
      bsplit(T, T.g[gi][j], eps * T.logb[j], T.gsp[gi], j);
    if (!sync()) break;
    // g_1 = f_0^{C,eps} (Algorithm 4.1 line 3 at the first iteration)
    {
      float v[2] = {0.f, 0.f};
      bcol_pass(T, c0, c1, gi, eps, k2, false, v, sh);
      publishf(v, 0);
      if (!sync()) break;
      if (gsum(1) > 0.0) {
        status = 3;
        break;
      }
      gi ^= 1;
    }
    double tol = last ? T.tol_last : T.tol_level;
    iter = 0;
    for (;;) {
      float u[2] = {0.f, 0.f};
      brow_pass(T, r0, r1, gi, eps, k2, false, u);   // f_k = g_k^{C,eps} (its numeric flags)
      u[0] = 0.f;
      if (!sync()) break;
      bcol_pass(T, c0, c1, gi, eps, k2, false, u, sh);   // f_k^{C,eps} and the L1 test
      publishf(u, 0);
      if (!sync()) break;
      const double l1 = gsum(0);
      ++iter;
      ++total;
      if (gsum(1) > 0.0) {
        status = 3;
        break;
      }
      col_l1 = l1;
      if (l1 < tol) {
        if (!last) break;
        // verify the pair (f_k, g_k): the row term of the L1 error
        float e[2] = {0.f, 0.f};
        brow_pass(T, r0, r1, gi, eps, k2, true, e);
        publishf(e, 8);
        if (!sync()) break;
        row_l1 = gsum(8);
        have_row = true;
        ++verify_rounds;
        if (row_l1 + col_l1 < T.tol_verify || verify_rounds >= 4) break;
        tol = 0.9 * (T.tol_verify - row_l1);
        if (!(tol > 0.0)) tol = 0.1 * T.tol_verify;
        have_row = false;
        continue;
      }
      if (iter >= T.max_iter) {
        status = 2;
        break;
      }
      gi ^= 1;   // commit g_{k+1} = f_k^{C,eps}
    }
  }
  const int levels = lev;
  if (status == 0) status = 1;
  if (status != 4) {
    // scores of the returned pair (f, g[gi]) at the last eps (the column
    // log-ratios are those of the last column pass)
    const double eps = T.eps[max(0, min(levels, T.nlev) - 1)];
    const float k2 = (float)(1.0 / (eps * 0.6931471805599453));
    if (!have_row) {
      float e[2] = {0.f, 0.f};
      brow_pass(T, r0, r1, gi, eps, k2, true, e);
      publishf(e, 8);
      if (sync()) row_l1 = gsum(8);
    }
    // float64 sums: <f,a>, sum pi, <pi1-a,f> | <g,b>, <pi^T1-b,g>, column L1,
    // <h,b> with h = f^{C,eps} from the last column half-step (other buffer)
    double v[4] = {0.0, 0.0, 0.0, 0.0}, u[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = r0 + threadIdx.x; i < r1; i += kBThreads) {
      const double e = (double)expm1f(T.Lrow[i]), ai = T.a[i], fi = T.f[i];
      v[0] += ai * fi;
      v[1] += ai * (1.0 + e);
      v[2] += ai * e * fi;
    }
    for (int j = c0 + threadIdx.x; j < c1; j += kBThreads) {
      const double e = (double)expm1f(T.Lcol[j]), bj = T.b[j], gj = T.g[gi][j];
      u[0] += bj * gj;
      u[1] += bj * e * gj;
      u[2] += bj * fabs(e);
      u[3] += bj * T.g[1 - gi][j];
    }
    if (status != 4 && sync()) {   // every rank has read the partials above
      publish(v, 0);
      publish(u, 12);
    }
    if (status != 4 && sync()) {
      const double fa = gsum(0), sumpi = gsum(1), gap_f = gsum(2);
      const double gb = gsum(12), gap_g = gsum(13), cl1 = gsum(14), sum_bh = gsum(15);
      const double c = 0.5 * (gb - fa);
      for (int i = r0 + threadIdx.x; i < r1; i += kBThreads) T.f_out[i] = T.f[i] + c;
      for (int j = c0 + threadIdx.x; j < c1; j += kBThreads) T.g_out[j] = T.g[gi][j] - c;
      if (rank == 0 && threadIdx.x == 0) {
        BatchOut* o = T.out;
        o->row_l1 = row_l1;
        o->col_l1 = cl1;
        o->q_dual = fa + gb - eps * (sumpi - 1.0);
        o->q_semi = fa + sum_bh;
        o->dual_gap = gap_f + gap_g + eps * (sumpi - 1.0);
        o->gauge = c;
      }
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
    brun_task(tasks[e.x], e.y, sh);
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
        double v = P.givenC ? (double)P.Cin[(size_t)i * P.m + j]
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

}  // namespace eotk
