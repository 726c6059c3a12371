// Persistent, shared-memory-staged log-sum-exp passes over a stored float32
// cost: the Sinkhorn half-steps of Eq. SK_iterations (paper Eq. foc_f and
// Eq. foc_g) and the trial and evaluation passes of Algorithm 4.1, for
// m % 4 == 0 and a 16-byte aligned cost.  Same inputs, outputs and modes as
// the striped passes of passes.cu; only the schedule and the arithmetic
// differ.
//
// Work decomposition (stream-K).  The cost is cut into tiles of 32 rows x 128
// columns, numbered output-block-major: for the column pass tile t lies in
// column block b = t / ntr (128 columns), row tile t % ntr; for the row pass in
// row block b = t / ntc (32 rows), column tile t % ntc.  A grid of G CTAs (the
// number the SMs hold at once: one wave) takes the contiguous chunks
// [floor(k T / G), floor((k+1) T / G)) of the T tiles, so every CTA streams
// the same number of bytes (+-1 tile) whatever the shape.  A chunk that covers
// only part of an output block leaves a partial (reference, sum) state per
// index in a [block][contributor][index] buffer; the last contributor of the
// block (atomic arrival counter) merges the contributors in a fixed order and
// finishes the block, so the results do not depend on scheduling.
//
// Pipeline.  One producer warp copies each tile row (<= 512 bytes) and the
// tile's reduction-side coefficients into a ring of four shared-memory stages
// with cp.async.bulk, completing on the stage's mbarrier; eight consumer warps
// reduce the tile and release the stage.  Every wait is bounded: a wait that
// gives up flags a numeric error and the kernel drains its copies and returns.
//
// Arithmetic per element, with the potentials split as described in
// eot_device.cuh (A = H(u) + M, K = M - H(s), AL / KL the low parts):
//     a = A_red - K_out                 exact (both in one binade)
//     t = a - C                         one rounding, relative to t
//     y = t * k2 + (AL_red + KL_out) * k2        exponent in log2 units
// two elements at a time with the packed float32x2 instructions, then exp2 on
// the MUFU and a packed accumulation.  The running sum of an output index is
// kept relative to an integer reference (log2 units) that stays 0 while the
// running maximum lies within 2^+-64 of the output potential's shift (the
// common case near a fixed point, where the sums are marginal ratios close to
// one) and is moved with an exact power-of-two rescaling otherwise.
#include "eot_device.cuh"
#include "eot_internal.h"
#include "pass_common.cuh"
#include "reduce.cuh"
#include "tc.cuh"

namespace eotk {

constexpr int kStR = 32;                                   // tile rows
constexpr int kStC = 128;                                  // tile columns
constexpr int kStStages = 4;
constexpr int kStTileBytes = kStR * kStC * 4;              // 16 KB
constexpr int kStStageBytes = kStTileBytes + 2 * kStC * 4; // + coefficient hi / lo
constexpr int kStSmem = kStStages * kStStageBytes;
constexpr int kStConsumers = 256;
constexpr int kStThreads = kStConsumers + 32;
constexpr int kStWait = 1 << 22;
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

// CTA whose chunk holds tile t (chunks [floor(kT/G), floor((k+1)T/G)), G <= T).
__device__ __forceinline__ int st_owner(long long t, long long T, int G) {
  return (int)(((t + 1) * (long long)G - 1) / T);
}

// Sum of three doubles over the 256 consumer threads; valid in thread 0.
__device__ __forceinline__ void cons_sum3(double v[3], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double x = warp_sum_d(v[k]);
    if (lane == 0) sh[k * 8 + wid] = x;
  }
  cons_sync();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += sh[k * 8 + w];
      v[k] = t;
    }
  }
  cons_sync();
}

// Sum of nblk per-block accumulators (stride 4) in a fixed order by the 256
// consumer threads; result valid in every consumer thread.
__device__ __forceinline__ void cons_grid_sum3(const double* __restrict__ acc, int nblk,
                                               double out[3], double* sh) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += kStConsumers) {
    v[0] += __ldcg(&acc[b * 4 + 0]);
    v[1] += __ldcg(&acc[b * 4 + 1]);
    v[2] += __ldcg(&acc[b * 4 + 2]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double x = warp_sum_d(v[k]);
    if (lane == 0) sh[k * 8 + wid] = x;
  }
  cons_sync();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[k * 8 + w];
    out[k] = t;
  }
  cons_sync();
}

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

__device__ __forceinline__ float2 ex2_2(float2 y) {
  return make_float2(ex2_approx(y.x), ex2_approx(y.y));
}

// Move the reference of one running sum when its running maximum rr (relative
// to the reference) left the window; returns the shift d (0 if none).
__device__ __forceinline__ float recentre(float& rr, float& ref, float& S) {
  if (fabsf(rr) <= kStWindow || !(rr > -INFINITY)) return 0.f;
  const float d = rintf(rr);
  S = scale2(S, -d);
  ref += d;
  rr -= d;
  return d;
}

template <bool COL>
__global__ void __launch_bounds__(kStThreads, 2)
    stream_pass_kernel(const Prob* __restrict__ PP, int mode) {
  const Prob& P = *PP;
  State* st = P.st;
  if (mode != MODE_PLAIN && mode != MODE_EVAL && st->done) return;
  if (COL && mode == MODE_TRIAL && !st->nr_ok) return;
  const int cf = st->cur_f, cg = st->cur_g;
  // buffers (as in the striped passes): a trial column pass reads f' and is
  // shifted by h = f_k^{C,eps}
  int src_f = cf, sh_g = cg, dst_g = (cg + 1) % 3;
  if (COL && mode == MODE_TRIAL) {
    src_f = 1 - cf;
    sh_g = (cg + 1) % 3;
    dst_g = (cg + 2) % 3;
  }
  if (mode == MODE_EVAL) dst_g = -1;
  const Split red = COL ? P.rs[src_f] : P.cs[cg];
  const Split outs = COL ? P.cs[sh_g] : P.rs[cf];

  extern __shared__ __align__(1024) unsigned char st_smem[];
  __shared__ __align__(8) uint64_t full_bar[kStStages];
  __shared__ __align__(8) uint64_t empty_bar[kStStages];
  __shared__ float2 s_pc[COL ? 8 : 1][kStC];      // column pass: per-warp partials
  __shared__ float s_mr[8][kStC];                 // merged partial heads
  __shared__ double s_ms[8][kStC];                // merged partial sums
  __shared__ double s_red[24];
  __shared__ unsigned s_flag;
  __shared__ int s_err;

  const int n = P.n, m = P.m;
  const int ntr = (n + kStR - 1) / kStR, ntc = (m + kStC - 1) / kStC;
  const long long T = (long long)ntr * ntc;
  const int G = gridDim.x;
  const int nT = COL ? ntr : ntc;     // tiles per output block
  const int nblk = COL ? ntc : ntr;   // output blocks
  const int width = COL ? kStC : kStR;
  const int slots = COL ? P.sk_slots_col : P.sk_slots_row;
  float2* __restrict__ part = COL ? P.sk_part_col : P.sk_part_row;
  unsigned* __restrict__ cnt = COL ? P.sk_cnt_col : P.sk_cnt_row;
  double* __restrict__ bacc = COL ? P.sk_acc_col : P.sk_acc_row;
  const long long t0 = T * blockIdx.x / G, t1 = T * (blockIdx.x + 1) / G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t sbase = smem_addr(st_smem);

  if (tid == 0) {
    for (int s = 0; s < kStStages; ++s) {
      mbar_init(smem_addr(&full_bar[s]), 1);
      mbar_init(smem_addr(&empty_bar[s]), 8);
    }
    s_err = 0;
    mbar_init_fence();
  }
  __syncthreads();

  if (warp == 8) {
    // ---------------- producer ----------------
    int it = 0;
    bool ok = true;
    for (long long t = t0; t < t1; ++t, ++it) {
      const int s = it % kStStages;
      if (it >= kStStages &&
          !mbar_wait(smem_addr(&empty_bar[s]), ((it / kStStages) - 1) & 1, kStWait)) {
        ok = false;
        break;
      }
      const int b = (int)(t / nT), q = (int)(t - (long long)b * nT);
      const int r0 = COL ? q * kStR : b * kStR;
      const int c0 = COL ? b * kStC : q * kStC;
      const int rows = min(kStR, n - r0), cols = min(kStC, m - c0);
      // reduction-side coefficients: rows of the tile (column pass, rounded up
      // to 4 floats: the split arrays are padded) or its columns (row pass)
      const int ncoef = COL ? ((rows + 3) & ~3) : cols;
      const uint32_t fb = smem_addr(&full_bar[s]);
      const uint32_t dst = sbase + (uint32_t)(s * kStStageBytes);
      if (lane == 0) mbar_expect_tx(fb, (uint32_t)(rows * cols * 4 + 2 * ncoef * 4));
      __syncwarp();
      if (lane < rows)
        bulk_load(dst + (uint32_t)(lane * kStC * 4), P.C + (size_t)(r0 + lane) * m + c0,
                  (uint32_t)(cols * 4), fb);
      if (lane == 0) {
        const int off = COL ? r0 : c0;
        bulk_load(dst + kStTileBytes, red.A + off, (uint32_t)(ncoef * 4), fb);
        bulk_load(dst + kStTileBytes + kStC * 4, red.AL + off, (uint32_t)(ncoef * 4), fb);
      }
      __syncwarp();
    }
    if (!ok) {
      if (lane == 0) {
        atomicAdd(&st->numeric, 1);
        s_err = 1;
      }
    }
    // drain: the last copy issued into every stage has landed before exit
    const int issued = it;
    for (int s = 0; s < kStStages && s < issued; ++s) {
      const int last = s + ((issued - 1 - s) / kStStages) * kStStages;
      mbar_wait(smem_addr(&full_bar[s]), (last / kStStages) & 1, kStWait);
    }
    return;
  }

  // ---------------- consumers ----------------
  const float k2 = P.k2;
  const float2 k2v = f2(k2, k2);
  const float2 m1 = f2(-1.f, -1.f);
  // per-thread output indices: column pass, 4 columns lane*4 + c of the block;
  // row pass, 4 rows 4*warp + u of the block
  float2 nK01, nK23, cc01, cc23;      // -K and KL*k2 (column pass)
  float nKr[4], ccr[4];               // the same per row (row pass)
  float ref[4], rr[4];
  float2 Sa[4];                       // column pass: Sa[0] = (S0, S1), Sa[1] = (S2, S3)
  bool ref0 = true;
  bool werr = false;                  // this warp gave up waiting

  // finish this CTA's piece of output block b
  auto flush = [&](int b) {
    const int kf = st_owner((long long)b * nT, T, G);
    const int kl = st_owner((long long)(b + 1) * nT - 1, T, G);
    const int nc = kl - kf + 1;
    const int slot = (int)blockIdx.x - kf;
    if (COL) {
      s_pc[warp][lane * 4 + 0] = f2(ref[0], Sa[0].x);
      s_pc[warp][lane * 4 + 1] = f2(ref[1], Sa[0].y);
      s_pc[warp][lane * 4 + 2] = f2(ref[2], Sa[1].x);
      s_pc[warp][lane * 4 + 3] = f2(ref[3], Sa[1].y);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float rf = ref[u], ss = Sa[u].x + Sa[u].y;
        const bool uni = __all_sync(0xffffffffu, rf == __shfl_sync(0xffffffffu, rf, 0));
        if (uni) {
          ss = warp_sum_f(ss);
        } else {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float r2 = __shfl_xor_sync(0xffffffffu, rf, o);
            const float s2 = __shfl_xor_sync(0xffffffffu, ss, o);
            lse2_merge(rf, ss, r2, s2);
          }
        }
        if (lane == 0) {
          s_mr[0][warp * 4 + u] = rf;
          s_ms[0][warp * 4 + u] = (double)ss;
        }
      }
    }
    // s_err may be raised by the producer at any time: take one value for all
    if (cons_sync_or(*(volatile int*)&s_err)) return;
    float R = -INFINITY;
    double Sd = 0.0;
    const int idx = b * width + tid;            // output index of thread tid < width
    const int lim = COL ? m : n;
    if (tid < width) {
      if (COL) {
#pragma unroll
        for (int w = 0; w < 8; ++w) merge_d(R, Sd, s_pc[w][tid].x, s_pc[w][tid].y);
      } else {
        R = s_mr[0][tid];
        Sd = s_ms[0][tid];
      }
      if (nc > 1 && idx < lim)
        part[((size_t)b * slots + slot) * width + tid] = f2(R, (float)Sd);
    }
    if (nc > 1) {
      __threadfence();
      cons_sync();
      if (tid == 0) s_flag = (atomicAdd(&cnt[b], 1u) == (unsigned)(nc - 1)) ? 1u : 0u;
      cons_sync();
      if (!s_flag) return;
      __threadfence();
      // the contributors' partials, merged by 256 / width groups in parallel
      const int c = tid % width, h = tid / width, ng = kStConsumers / width;
      float Rg = -INFINITY;
      double Sg = 0.0;
      if (b * width + c < lim)
        merge_segments(part + (size_t)b * slots * width, nc, width, c, h, ng, Rg, Sg);
      s_mr[h][c] = Rg;
      s_ms[h][c] = Sg;
      cons_sync();
      if (tid < width) {
        R = s_mr[0][tid];
        Sd = s_ms[0][tid];
        for (int g = 1; g < ng; ++g) merge_dd(R, Sd, s_mr[g][tid], s_ms[g][tid]);
      }
      if (tid == 0) cnt[b] = 0u;
    }
    double accv[3] = {0.0, 0.0, 0.0};
    if (tid < width && idx < lim) {
      double* out;
      Split so;
      if (mode == MODE_PLAIN) {
        out = P.out_plain;
        so = Split{nullptr, nullptr, nullptr, nullptr};
      } else if (mode == MODE_EVAL) {
        out = nullptr;
        so = Split{nullptr, nullptr, nullptr, nullptr};
      } else if (COL) {
        out = P.g[dst_g];
        so = P.cs[dst_g];
      } else {
        out = P.f[cf];
        so = P.rs[cf];
      }
      if (COL) {
        finish_index(R, Sd, idx, P, P.g[sh_g], P.b, P.logb, out, so, P.Lcol, accv, &st->numeric);
        if (mode == MODE_PLAIN && P.logratio_plain) P.logratio_plain[idx] = (double)P.Lcol[idx];
      } else {
        finish_index(R, Sd, idx, P, P.f[cf], P.a, P.loga, out, so, P.Lrow, accv, &st->numeric);
        if (mode == MODE_PLAIN && P.logratio_plain) P.logratio_plain[idx] = (double)P.Lrow[idx];
      }
    }
    cons_sum3(accv, s_red);
    if (tid == 0) {
      double* ab = bacc + b * 4;
      ab[0] = accv[0];
      ab[1] = accv[1];
      ab[2] = accv[2];
      __threadfence();
      s_flag = (atomicAdd(&P.gcnt[COL ? 0 : 1], 1u) == (unsigned)(nblk - 1)) ? 1u : 0u;
    }
    cons_sync();
    if (!s_flag) return;
    __threadfence();
    double tot[3];
    cons_grid_sum3(bacc, nblk, tot, s_red);
    if (tid == 0) {
      P.gcnt[COL ? 0 : 1] = 0u;
      if (COL) final_step(P, mode, tot, dst_g);
      else if (mode == MODE_EVAL) st->l1_row = tot[0];
      else final_step(P, mode == MODE_PLAIN ? MODE_PLAIN : MODE_SK_ROW, tot, cf);
    }
  };

  auto start_block = [&](int b) {
    ref0 = true;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      ref[c] = 0.f;
      rr[c] = -INFINITY;
      Sa[c] = f2(0.f, 0.f);
    }
    if (COL) {
      float K[4], KL[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = b * kStC + lane * 4 + c;
        K[c] = j < m ? outs.K[j] : P.M;
        KL[c] = j < m ? outs.KL[j] : 0.f;
      }
      nK01 = f2(-K[0], -K[1]);
      nK23 = f2(-K[2], -K[3]);
      cc01 = f2(KL[0] * k2, KL[1] * k2);
      cc23 = f2(KL[2] * k2, KL[3] * k2);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = b * kStR + warp * 4 + u;
        nKr[u] = i < n ? -outs.K[i] : -P.M;
        ccr[u] = i < n ? outs.KL[i] * k2 : 0.f;
      }
    }
  };

  int cur_b = -1;
  int it = 0;
  for (long long t = t0; t < t1; ++t, ++it) {
    const int b = (int)(t / nT), q = (int)(t - (long long)b * nT);
    if (b != cur_b) {
      if (cur_b >= 0) flush(cur_b);
      cur_b = b;
      start_block(b);
    }
    const int s = it % kStStages;
    if (!werr && !mbar_wait(smem_addr(&full_bar[s]), (it / kStStages) & 1, kStWait)) {
      werr = true;
      if (lane == 0) {
        atomicAdd(&st->numeric, 1);
        s_err = 1;
      }
    }
    if (!werr) {
      const float* tile = reinterpret_cast<const float*>(st_smem + s * kStStageBytes);
      const float* cA = tile + kStR * kStC;
      const float* cAL = cA + kStC;
      const int r0 = COL ? q * kStR : b * kStR;
      const int c0 = COL ? b * kStC : q * kStC;
      const bool fullt = (r0 + kStR <= n) && (c0 + kStC <= m);
      float2 ya[4], yb[4];   // column pass: rows u, columns (0,1) / (2,3); row pass: row u
      if (COL) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = warp + 8 * u;
          const float4 cv = *reinterpret_cast<const float4*>(tile + r * kStC + lane * 4);
          const float ar = cA[r];
          const float al = cAL[r] * k2;
          const float2 arr = f2(ar, ar), all = f2(al, al);
          const float2 ta = __ffma2_rn(f2(cv.x, cv.y), m1, __fadd2_rn(arr, nK01));
          const float2 tb = __ffma2_rn(f2(cv.z, cv.w), m1, __fadd2_rn(arr, nK23));
          ya[u] = __ffma2_rn(ta, k2v, __fadd2_rn(all, cc01));
          yb[u] = __ffma2_rn(tb, k2v, __fadd2_rn(all, cc23));
        }
        if (!fullt) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const bool rv = r0 + warp + 8 * u < n;
            const int j = c0 + lane * 4;
            ya[u].x = (rv && j + 0 < m) ? ya[u].x : -INFINITY;
            ya[u].y = (rv && j + 1 < m) ? ya[u].y : -INFINITY;
            yb[u].x = (rv && j + 2 < m) ? yb[u].x : -INFINITY;
            yb[u].y = (rv && j + 3 < m) ? yb[u].y : -INFINITY;
          }
        }
        if (!ref0) {
          const float2 na = f2(-ref[0], -ref[1]), nb = f2(-ref[2], -ref[3]);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            ya[u] = __fadd2_rn(ya[u], na);
            yb[u] = __fadd2_rn(yb[u], nb);
          }
        }
        rr[0] = fmaxf(rr[0], fmaxf(fmaxf(ya[0].x, ya[1].x), fmaxf(ya[2].x, ya[3].x)));
        rr[1] = fmaxf(rr[1], fmaxf(fmaxf(ya[0].y, ya[1].y), fmaxf(ya[2].y, ya[3].y)));
        rr[2] = fmaxf(rr[2], fmaxf(fmaxf(yb[0].x, yb[1].x), fmaxf(yb[2].x, yb[3].x)));
        rr[3] = fmaxf(rr[3], fmaxf(fmaxf(yb[0].y, yb[1].y), fmaxf(yb[2].y, yb[3].y)));
        if (!(fabsf(rr[0]) <= kStWindow && fabsf(rr[1]) <= kStWindow &&
              fabsf(rr[2]) <= kStWindow && fabsf(rr[3]) <= kStWindow)) {
          const float d0 = recentre(rr[0], ref[0], Sa[0].x);
          const float d1 = recentre(rr[1], ref[1], Sa[0].y);
          const float d2 = recentre(rr[2], ref[2], Sa[1].x);
          const float d3 = recentre(rr[3], ref[3], Sa[1].y);
          const float2 na = f2(-d0, -d1), nb = f2(-d2, -d3);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            ya[u] = __fadd2_rn(ya[u], na);
            yb[u] = __fadd2_rn(yb[u], nb);
          }
          ref0 = ref[0] == 0.f && ref[1] == 0.f && ref[2] == 0.f && ref[3] == 0.f;
        }
        Sa[0] = __fadd2_rn(Sa[0], __fadd2_rn(__fadd2_rn(ex2_2(ya[0]), ex2_2(ya[1])),
                                             __fadd2_rn(ex2_2(ya[2]), ex2_2(ya[3]))));
        Sa[1] = __fadd2_rn(Sa[1], __fadd2_rn(__fadd2_rn(ex2_2(yb[0]), ex2_2(yb[1])),
                                             __fadd2_rn(ex2_2(yb[2]), ex2_2(yb[3]))));
      } else {
        const float4 ca = *reinterpret_cast<const float4*>(cA + lane * 4);
        const float4 cl = *reinterpret_cast<const float4*>(cAL + lane * 4);
        const float2 caa = f2(ca.x, ca.y), cab = f2(ca.z, ca.w);
        const float2 ala = __fmul2_rn(f2(cl.x, cl.y), k2v), alb = __fmul2_rn(f2(cl.z, cl.w), k2v);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = warp * 4 + u;
          const float4 cv = *reinterpret_cast<const float4*>(tile + r * kStC + lane * 4);
          const float2 nk = f2(nKr[u], nKr[u]), cc = f2(ccr[u], ccr[u]);
          const float2 ta = __ffma2_rn(f2(cv.x, cv.y), m1, __fadd2_rn(caa, nk));
          const float2 tb = __ffma2_rn(f2(cv.z, cv.w), m1, __fadd2_rn(cab, nk));
          ya[u] = __ffma2_rn(ta, k2v, __fadd2_rn(ala, cc));
          yb[u] = __ffma2_rn(tb, k2v, __fadd2_rn(alb, cc));
        }
        if (!fullt) {
          const int j = c0 + lane * 4;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const bool rv = r0 + warp * 4 + u < n;
            ya[u].x = (rv && j + 0 < m) ? ya[u].x : -INFINITY;
            ya[u].y = (rv && j + 1 < m) ? ya[u].y : -INFINITY;
            yb[u].x = (rv && j + 2 < m) ? yb[u].x : -INFINITY;
            yb[u].y = (rv && j + 3 < m) ? yb[u].y : -INFINITY;
          }
        }
        if (!ref0) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 nr = f2(-ref[u], -ref[u]);
            ya[u] = __fadd2_rn(ya[u], nr);
            yb[u] = __fadd2_rn(yb[u], nr);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          rr[u] = fmaxf(rr[u], fmaxf(fmaxf(ya[u].x, ya[u].y), fmaxf(yb[u].x, yb[u].y)));
        if (!(fabsf(rr[0]) <= kStWindow && fabsf(rr[1]) <= kStWindow &&
              fabsf(rr[2]) <= kStWindow && fabsf(rr[3]) <= kStWindow)) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            // the row's running sum is held as a pair: rescale both halves
            float sx = Sa[u].x, sy = Sa[u].y, rx = ref[u], rry = rr[u];
            const float d = recentre(rry, rx, sx);
            if (d != 0.f) {
              sy = scale2(sy, -d);
              ya[u] = __fadd2_rn(ya[u], f2(-d, -d));
              yb[u] = __fadd2_rn(yb[u], f2(-d, -d));
            }
            Sa[u] = f2(sx, sy);
            ref[u] = rx;
            rr[u] = rry;
          }
          ref0 = ref[0] == 0.f && ref[1] == 0.f && ref[2] == 0.f && ref[3] == 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          Sa[u] = __fadd2_rn(Sa[u], __fadd2_rn(ex2_2(ya[u]), ex2_2(yb[u])));
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive1(smem_addr(&empty_bar[s]));
  }
  if (cur_b >= 0) flush(cur_b);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
void init_stream_attributes() {
  cudaFuncSetAttribute(stream_pass_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kStSmem);
  cudaFuncSetAttribute(stream_pass_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kStSmem);
}

// CTAs of one wave of the stream kernels (per SM count), 0 if they cannot run.
int stream_ctas_per_sm() {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, stream_pass_kernel<true>, kStThreads,
                                                    kStSmem) != cudaSuccess)
    a = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, stream_pass_kernel<false>, kStThreads,
                                                    kStSmem) != cudaSuccess)
    b = 0;
  cudaGetLastError();
  return a < b ? a : b;
}

// Grid size and contributor slots of one stream pass over an n x m cost.
void stream_plan(int n, int m, bool col, int ctas, int* grid, int* slots) {
  const long long ntr = (n + kStR - 1) / kStR, ntc = (m + kStC - 1) / kStC;
  const long long T = ntr * ntc;
  long long G = ctas;
  if (G > T) G = T;
  if (G < 1) G = 1;
  const long long nT = col ? ntr : ntc, nblk = col ? ntc : ntr;
  long long mx = 1;
  for (long long b = 0; b < nblk; ++b) {
    const long long kf = ((b * nT + 1) * G - 1) / T;
    const long long kl = (((b + 1) * nT) * G - 1) / T;
    if (kl - kf + 1 > mx) mx = kl - kf + 1;
  }
  *grid = (int)G;
  *slots = (int)mx;
}

cudaError_t launch_stream_pass(const Prob* dP, const Prob& hP, bool col, int mode,
                               cudaStream_t s) {
  if (col)
    stream_pass_kernel<true><<<hP.sk_gcol, kStThreads, kStSmem, s>>>(dP, mode);
  else
    stream_pass_kernel<false><<<hP.sk_grow, kStThreads, kStSmem, s>>>(dP, mode);
  return cudaGetLastError();
}

}  // namespace eotk
