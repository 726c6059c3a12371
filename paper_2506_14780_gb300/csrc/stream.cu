// Persistent, shared-memory-staged log-sum-exp passes over a stored float32
// cost: the Sinkhorn half-steps of Eq. SK_iterations (paper Eq. foc_f and
// Eq. foc_g) and the trial and evaluation passes of Algorithm 4.1, for
// m % 4 == 0 and a 16-byte aligned cost.  Same inputs, outputs and modes as
// the striped passes of passes.cu; only the schedule and the arithmetic
// differ.  Two kernels share the code below:
//   * stream_pass_kernel: one half-step per launch (any mode); the last
//     contributor of an output block finishes it;
//   * sk_coop_kernel: whole log-domain Sinkhorn iterations (row then column
//     half-step, Eq. SK_iterations) in one cooperative launch, the phases
//     separated by grid barriers and the output blocks finished by all CTAs
//     in parallel, until the L1 test of Algorithm 4.1 passes.
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
// Pipeline.  One lane of a producer warp loads each tile with one tiled tensor
// copy (TMA, 2-D map of C) and the tile's reduction-side coefficients with two
// bulk copies into a ring of four shared-memory stages, completing on the
// stage's mbarrier; eight consumer warps reduce the tile and release the
// stage.  Every wait (stages, grid barriers) is bounded: a wait that gives up
// flags a numeric error and the kernel drains its copies and returns.
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
// one); otherwise it follows the running maximum (see move_ref), with an exact
// power-of-two rescaling of the sum and the terms re-formed from the raw
// exponents, so that the reference never costs the dominant terms precision.
#include "eot_device.cuh"
#include "eot_internal.h"
#include "pass_common.cuh"
#include "reduce.cuh"
#include "tc.cuh"
#include "stream_common.cuh"

namespace eotk {

constexpr int kStR = 32;                                   // tile rows
constexpr int kStC = 128;                                  // tile columns
constexpr int kStStages = 4;
constexpr int kStTileBytes = kStR * kStC * 4;              // 16 KB
constexpr int kStStageBytes = kStTileBytes + 2 * kStC * 4; // + coefficient hi / lo
constexpr int kStSmem = kStStages * kStStageBytes;
constexpr int kStThreads = kStConsumers + 32;
constexpr int kStWait = 1 << 22;
constexpr int kStPend = 16;

// Static shared state of a stream CTA.
struct StShared {
  uint64_t full_bar[kStStages];
  uint64_t empty_bar[kStStages];
  float2 pc[8][kStC];     // column pass: per-warp partials
  float mr[8][kStC];      // merged partial heads
  double ms[8][kStC];     // merged partial sums
  double red[24];
  unsigned flag;
  int err;
  int pend[kStPend];      // blocks this CTA finishes after its stream
  int npend;
  int done;               // cooperative kernel: decision of the last iteration
};

// Tile geometry of the n x m cost and the chunks of a grid of G CTAs.
struct StGeom {
  int n, m, ntr, ntc, G;
  long long T;
  __device__ StGeom(int n_, int m_, int G_)
      : n(n_), m(m_), ntr((n_ + kStR - 1) / kStR), ntc((m_ + kStC - 1) / kStC), G(G_) {
    T = (long long)ntr * ntc;
  }
  __device__ int nT(bool col) const { return col ? ntr : ntc; }      // tiles per block
  __device__ int nblk(bool col) const { return col ? ntc : ntr; }    // output blocks
  __device__ long long first(int k) const { return T * k / G; }
  __device__ void tile(bool col, long long t, int& b, int& q, int& r0, int& c0,
                       int& ncoef) const {
    const int nt = nT(col);
    b = (int)(t / nt);
    q = (int)(t - (long long)b * nt);
    r0 = col ? q * kStR : b * kStR;
    c0 = col ? b * kStC : q * kStC;
    const int rows = min(kStR, n - r0), cols = min(kStC, m - c0);
    // reduction-side coefficients: rows of the tile (column pass, rounded up
    // to 4 floats: the split arrays are padded) or its columns (row pass)
    ncoef = col ? ((rows + 3) & ~3) : cols;
  }
  __device__ void contributors(bool col, int b, int& kf, int& nc) const {
    const int nt = nT(col);
    kf = st_owner((long long)b * nt, T, G);
    nc = st_owner((long long)(b + 1) * nt - 1, T, G) - kf + 1;
  }
};

// Producer warp: tiles [t0, t1) of this CTA into the ring, `it` the ring
// position of t0.  The cost copies of the first `npre` tiles were issued
// already (with their byte counts); their coefficients are added here.
template <bool COL>
__device__ bool st_produce(const Prob* PP, const StGeom& g, const PassIo& io, StShared& sh,
                           uint32_t sbase, long long t0, long long t1, int it, int npre) {
  const int lane = threadIdx.x & 31;
  for (long long t = t0; t < t1; ++t, ++it) {
    const int s = it % kStStages;
    const bool pre = (t - t0) < npre;
    if (!pre && it >= kStStages &&
        !mbar_wait(smem_addr(&sh.empty_bar[s]), ((it / kStStages) - 1) & 1, kStWait))
      return false;
    int b, q, r0, c0, ncoef;
    g.tile(COL, t, b, q, r0, c0, ncoef);
    const uint32_t fb = smem_addr(&sh.full_bar[s]);
    const uint32_t dst = sbase + (uint32_t)(s * kStStageBytes);
    if (lane == 0) {
      if (!pre) {
        mbar_expect_tx(fb, (uint32_t)(kStTileBytes + 2 * ncoef * 4));
        // c0 is a multiple of 128 columns: the box starts on a 16-byte boundary
        tma_load_2d(dst, &PP->tmC, c0, r0, fb);
      }
      const int off = COL ? r0 : c0;
      bulk_load(dst + kStTileBytes, io.red.A + off, (uint32_t)(ncoef * 4), fb);
      bulk_load(dst + kStTileBytes + kStC * 4, io.red.AL + off, (uint32_t)(ncoef * 4), fb);
    }
    __syncwarp();
  }
  return true;
}

// Wait until the last copy issued into every stage has landed (before exit).
__device__ __forceinline__ void st_drain(StShared& sh, int issued) {
  for (int s = 0; s < kStStages && s < issued; ++s) {
    const int last = s + ((issued - 1 - s) / kStStages) * kStStages;
    mbar_wait(smem_addr(&sh.full_bar[s]), (last / kStStages) & 1, kStWait);
  }
}

// Finish output block b from its contributors' partials: potentials, split
// arrays, log-ratios, and the block's three sums in bacc[b].  With last_step,
// the block's arrival on the grid counter and, for the last block, the
// grid-wide step of the mode.  Called by the 256 consumer threads.
template <bool COL>
__device__ void st_finish_block(const Prob& P, const StGeom& g, const PassIo& io, StShared& sh,
                                int b, bool last_step) {
  State* st = P.st;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int width = COL ? kStC : kStR;
  const int slots = COL ? P.sk_slots_col : P.sk_slots_row;
  const float2* part = COL ? P.sk_part_col : P.sk_part_row;
  unsigned* cnt = COL ? P.sk_cnt_col : P.sk_cnt_row;
  double* bacc = COL ? P.sk_acc_col : P.sk_acc_row;
  const int lim = COL ? g.m : g.n;
  const int nblk = g.nblk(COL);
  const int mode = io.mode;
  int kf, nc;
  g.contributors(COL, b, kf, nc);
  // the contributors' partials, merged by 256 / width groups in parallel
  const int c = tid % width, h = tid / width, ng = kStConsumers / width;
  float Rg = -INFINITY;
  double Sg = 0.0;
  if (b * width + c < lim)
    merge_segments(part + (size_t)b * slots * width, nc, width, c, h, ng, Rg, Sg);
  sh.mr[h][c] = Rg;
  sh.ms[h][c] = Sg;
  cons_sync();
  const int idx = b * width + tid;            // output index of thread tid < width
  float R = -INFINITY;
  double Sd = 0.0;
  if (tid < width) {
    R = sh.mr[0][tid];
    Sd = sh.ms[0][tid];
    for (int gg = 1; gg < ng; ++gg) merge_dd(R, Sd, sh.mr[gg][tid], sh.ms[gg][tid]);
  }
  if (tid == 0) cnt[b] = 0u;
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
      out = P.g[io.dst_g];
      so = P.cs[io.dst_g];
    } else {
      out = P.f[io.cf];
      so = P.rs[io.cf];
    }
    if (COL) {
      finish_index(R, Sd, idx, P, P.g[io.sh_g], P.b, P.logb, out, so, P.Lcol, accv, &st->numeric);
      if (mode == MODE_PLAIN && P.logratio_plain) P.logratio_plain[idx] = (double)P.Lcol[idx];
    } else {
      finish_index(R, Sd, idx, P, P.f[io.cf], P.a, P.loga, out, so, P.Lrow, accv, &st->numeric);
      if (mode == MODE_PLAIN && P.logratio_plain) P.logratio_plain[idx] = (double)P.Lrow[idx];
    }
  }
  cons_sum3(accv, sh.red, width < 32 ? 32 : width);
  if (tid == 0) {
    double* ab = bacc + b * 4;
    ab[0] = accv[0];
    ab[1] = accv[1];
    ab[2] = accv[2];
    if (last_step)
      sh.flag = (arrive_count(&P.gcnt[COL ? 0 : 1]) == (unsigned)(nblk - 1)) ? 1u : 0u;
  }
  cons_sync();
  if (!last_step || !sh.flag) return;
  if (warp == 0) {
    double tot[3];
    warp0_grid_sum3(bacc, nblk, tot);
    if (tid == 0) {
      P.gcnt[COL ? 0 : 1] = 0u;
      if (COL) final_step(P, mode, tot, io.dst_g);
      else if (mode == MODE_EVAL) st->l1_row = tot[0];
      else final_step(P, mode == MODE_PLAIN ? MODE_PLAIN : MODE_SK_ROW, tot, io.cf);
    }
  }
}

// Producer: cost copies (with the stage's byte count) of the first `npre`
// tiles of a coming phase, issued ahead of the grid barriers; the phase's
// st_produce adds their coefficients.  Returns how many were issued.
template <bool COL>
__device__ int st_prefetch(const Prob* PP, const StGeom& g, StShared& sh, uint32_t sbase,
                           long long t0, int npre, int it) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < npre; ++k, ++it) {
    const int s = it % kStStages;
    if (it >= kStStages &&
        !mbar_wait(smem_addr(&sh.empty_bar[s]), ((it / kStStages) - 1) & 1, kStWait))
      return k;
    int b, q, r0, c0, ncoef;
    g.tile(COL, t0 + k, b, q, r0, c0, ncoef);
    if (lane == 0) {
      const uint32_t fb = smem_addr(&sh.full_bar[s]);
      mbar_expect_tx(fb, (uint32_t)(kStTileBytes + 2 * ncoef * 4));
      tma_load_2d(sbase + (uint32_t)(s * kStStageBytes), &PP->tmC, c0, r0, fb);
    }
    __syncwarp();
  }
  return npre;
}

// Consumer warps: reduce tiles [t0, t1) of this CTA (`it` the ring position
// of t0), publish the partial state of every output block piece with an
// arrival on the block's counter, and finish the blocks this CTA arrived last
// on after the stream.  With `coop` (cooperative loop) a finished block only
// leaves its sums (the grid barrier that follows does the rest); otherwise the
// last block also takes the grid-wide step of the mode.
template <bool COL>
__device__ void st_consume(const Prob& P, const StGeom& g, const PassIo& io, StShared& sh,
                           const unsigned char* st_smem, long long t0, long long t1, int it,
                           bool coop) {
  State* st = P.st;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = g.n, m = g.m;
  const int width = COL ? kStC : kStR;
  const int slots = COL ? P.sk_slots_col : P.sk_slots_row;
  float2* __restrict__ part = COL ? P.sk_part_col : P.sk_part_row;
  unsigned* __restrict__ cnt = COL ? P.sk_cnt_col : P.sk_cnt_row;
  const int lim = COL ? m : n;
  const float k2 = P.k2;
  const float2 k2v = f2(k2, k2);
  const float2 m1 = f2(-1.f, -1.f);
  // per-thread output indices: column pass, 4 columns lane*4 + c of the block;
  // row pass, 4 rows 4*warp + u of the block
  float2 nK01, nK23, cc01, cc23;      // -K and KL*k2 (column pass)
  float nKr[4], ccr[4];               // the same per row (row pass)
  float ref[4] = {0.f, 0.f, 0.f, 0.f}, rr[4];
  float2 Sa[4] = {};                  // column pass: Sa[0] = (S0, S1), Sa[1] = (S2, S3)
  float2 Ca[2] = {};                  // column pass: their compensations
  bool ref0 = true;
  bool werr = false;                  // this warp gave up waiting

  auto finish_list = [&]() {
    const int np = sh.npend;
    for (int k = 0; k < np; ++k) st_finish_block<COL>(P, g, io, sh, sh.pend[k], !coop);
    cons_sync();
    if (tid == 0) sh.npend = 0;
  };

  auto publish = [&](int b) {
    if (COL) {
      kahan_fold2(Sa[0], Ca[0]);
      kahan_fold2(Sa[1], Ca[1]);
      sh.pc[warp][lane * 4 + 0] = f2(ref[0], Sa[0].x);
      sh.pc[warp][lane * 4 + 1] = f2(ref[1], Sa[0].y);
      sh.pc[warp][lane * 4 + 2] = f2(ref[2], Sa[1].x);
      sh.pc[warp][lane * 4 + 3] = f2(ref[3], Sa[1].y);
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
          sh.mr[0][warp * 4 + u] = rf;
          sh.ms[0][warp * 4 + u] = (double)ss;
        }
      }
    }
    // sh.err may be raised by the producer at any time: take one value for all
    if (cons_sync_or(*(volatile int*)&sh.err)) return;
    if (sh.npend == kStPend) finish_list();   // the list is full (tiny blocks)
    int kf, nc;
    g.contributors(COL, b, kf, nc);
    const int idx = b * width + tid;
    if (tid < width) {
      float R = -INFINITY;
      double Sd = 0.0;
      if (COL) {
#pragma unroll
        for (int w = 0; w < 8; ++w) merge_d(R, Sd, sh.pc[w][tid].x, sh.pc[w][tid].y);
      } else {
        R = sh.mr[0][tid];
        Sd = sh.ms[0][tid];
      }
      if (idx < lim && EOT_CHECK((int)blockIdx.x - kf >= 0 && (int)blockIdx.x - kf < slots, 301))
        part[((size_t)b * slots + ((int)blockIdx.x - kf)) * width + tid] = f2(R, (float)Sd);
    }
    cons_sync();
    if (tid == 0 && arrive_count(&cnt[b]) == (unsigned)(nc - 1)) sh.pend[sh.npend++] = b;
  };

  auto start_block = [&](int b) {
    ref0 = true;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      ref[c] = 0.f;
      rr[c] = -INFINITY;
      Sa[c] = f2(0.f, 0.f);
      if (c < 2) Ca[c] = f2(0.f, 0.f);
    }
    if (COL) {
      float K[4], KL[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = b * kStC + lane * 4 + c;
        K[c] = j < m ? io.outs.K[j] : P.M;
        KL[c] = j < m ? io.outs.KL[j] : 0.f;
      }
      nK01 = f2(-K[0], -K[1]);
      nK23 = f2(-K[2], -K[3]);
      cc01 = f2(KL[0] * k2, KL[1] * k2);
      cc23 = f2(KL[2] * k2, KL[3] * k2);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = b * kStR + warp * 4 + u;
        nKr[u] = i < n ? -io.outs.K[i] : -P.M;
        ccr[u] = i < n ? io.outs.KL[i] * k2 : 0.f;
      }
    }
  };

  int cur_b = -1;
  for (long long t = t0; t < t1; ++t, ++it) {
    int b, q, r0, c0, ncoef;
    g.tile(COL, t, b, q, r0, c0, ncoef);
    if (b != cur_b) {
      if (cur_b >= 0) publish(cur_b);
      cur_b = b;
      start_block(b);
    }
    const int s = it % kStStages;
    if (!werr && !mbar_wait(smem_addr(&sh.full_bar[s]), (it / kStStages) & 1, kStWait)) {
      werr = true;
      if (lane == 0) {
        atomicAdd(&st->numeric, 1);
        sh.err = 1;
      }
    }
    if (!werr) {
      const float* tile = reinterpret_cast<const float*>(st_smem + s * kStStageBytes);
      const float* cA = tile + kStR * kStC;
      const float* cAL = cA + kStC;
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
        // z = y - ref (the raw exponents y are kept for a change of reference)
        float2 za[4], zb[4];
        const float2 na = f2(-ref[0], -ref[1]), nb = f2(-ref[2], -ref[3]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          za[u] = ref0 ? ya[u] : __fadd2_rn(ya[u], na);
          zb[u] = ref0 ? yb[u] : __fadd2_rn(yb[u], nb);
        }
        rr[0] = fmaxf(rr[0], fmaxf(fmaxf(za[0].x, za[1].x), fmaxf(za[2].x, za[3].x)));
        rr[1] = fmaxf(rr[1], fmaxf(fmaxf(za[0].y, za[1].y), fmaxf(za[2].y, za[3].y)));
        rr[2] = fmaxf(rr[2], fmaxf(fmaxf(zb[0].x, zb[1].x), fmaxf(zb[2].x, zb[3].x)));
        rr[3] = fmaxf(rr[3], fmaxf(fmaxf(zb[0].y, zb[1].y), fmaxf(zb[2].y, zb[3].y)));
        const bool move = ref0 ? !(fabsf(rr[0]) <= kStWindow && fabsf(rr[1]) <= kStWindow &&
                                   fabsf(rr[2]) <= kStWindow && fabsf(rr[3]) <= kStWindow)
                               : (needs_move(rr[0], ref[0]) || needs_move(rr[1], ref[1]) ||
                                  needs_move(rr[2], ref[2]) || needs_move(rr[3], ref[3]));
        if (move) {
          kahan_fold2(Sa[0], Ca[0]);
          kahan_fold2(Sa[1], Ca[1]);
          move_ref(rr[0], ref[0], Sa[0].x);
          move_ref(rr[1], ref[1], Sa[0].y);
          move_ref(rr[2], ref[2], Sa[1].x);
          move_ref(rr[3], ref[3], Sa[1].y);
          ref0 = ref[0] == 0.f && ref[1] == 0.f && ref[2] == 0.f && ref[3] == 0.f;
          const float2 ma = f2(-ref[0], -ref[1]), mb = f2(-ref[2], -ref[3]);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            za[u] = __fadd2_rn(ya[u], ma);
            zb[u] = __fadd2_rn(yb[u], mb);
          }
        }
        kahan_add2(Sa[0], Ca[0], __fadd2_rn(__fadd2_rn(ex2_2(za[0]), ex2_2(za[1])),
                                            __fadd2_rn(ex2_2(za[2]), ex2_2(za[3]))));
        kahan_add2(Sa[1], Ca[1], __fadd2_rn(__fadd2_rn(ex2_2(zb[0]), ex2_2(zb[1])),
                                            __fadd2_rn(ex2_2(zb[2]), ex2_2(zb[3]))));
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
        float2 za[4], zb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 nr = f2(-ref[u], -ref[u]);
          za[u] = ref0 ? ya[u] : __fadd2_rn(ya[u], nr);
          zb[u] = ref0 ? yb[u] : __fadd2_rn(yb[u], nr);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          rr[u] = fmaxf(rr[u], fmaxf(fmaxf(za[u].x, za[u].y), fmaxf(zb[u].x, zb[u].y)));
        const bool move = ref0 ? !(fabsf(rr[0]) <= kStWindow && fabsf(rr[1]) <= kStWindow &&
                                   fabsf(rr[2]) <= kStWindow && fabsf(rr[3]) <= kStWindow)
                               : (needs_move(rr[0], ref[0]) || needs_move(rr[1], ref[1]) ||
                                  needs_move(rr[2], ref[2]) || needs_move(rr[3], ref[3]));
        if (move) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            // the row's running sum is held as a pair: rescale both halves
            float sx = Sa[u].x, rx = ref[u], rry = rr[u];
            const float old = rx;
            move_ref(rry, rx, sx);
            Sa[u] = f2(sx, rx != old ? scale2(Sa[u].y, old - rx) : Sa[u].y);
            ref[u] = rx;
            rr[u] = rry;
            const float2 nr = f2(-rx, -rx);
            za[u] = __fadd2_rn(ya[u], nr);
            zb[u] = __fadd2_rn(yb[u], nr);
          }
          ref0 = ref[0] == 0.f && ref[1] == 0.f && ref[2] == 0.f && ref[3] == 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          Sa[u] = __fadd2_rn(Sa[u], __fadd2_rn(ex2_2(za[u]), ex2_2(zb[u])));
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive1(smem_addr(&sh.empty_bar[s]));
  }
  // the stream is done: the next kernel may start its prologue
  if (!coop) pdl_trigger();
  if (cur_b >= 0) publish(cur_b);
  if (!cons_sync_or(*(volatile int*)&sh.err)) finish_list();
}

__device__ __forceinline__ void st_init_shared(StShared& sh) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStStages; ++s) {
      mbar_init(smem_addr(&sh.full_bar[s]), 1);
      mbar_init(smem_addr(&sh.empty_bar[s]), 8);
    }
    sh.err = 0;
    sh.npend = 0;
    sh.done = 0;
    mbar_init_fence();
  }
  __syncthreads();
}

// One half-step of any mode (one launch).
template <bool COL>
__global__ void __launch_bounds__(kStThreads, 2)
    stream_pass_kernel(const Prob* __restrict__ PP, int mode) {
  // PP->tmC is read by the tensor-copy unit: PP points to global memory.  The
  // problem description (*PP) and the cost are not written by the kernels of
  // a solve, so they are read before the programmatic-launch wait; the state
  // and the potentials only after it.
  const Prob& P = *PP;
  State* st = P.st;
  extern __shared__ __align__(1024) unsigned char st_smem[];
  __shared__ StShared sh;
  const StGeom g(P.n, P.m, (int)gridDim.x);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = smem_addr(st_smem);
  const long long t0 = g.first(blockIdx.x), t1 = g.first(blockIdx.x + 1);
  st_init_shared(sh);
  // The first stages of the cost tiles do not depend on the preceding kernel:
  // start them before waiting for it (they complete when the coefficients
  // are added).
  const int npre = (int)min((long long)kStStages, t1 - t0);
  if (warp == 8 && lane == 0) {
    for (int it = 0; it < npre; ++it) {
      int b, q, r0, c0, ncoef;
      g.tile(COL, t0 + it, b, q, r0, c0, ncoef);
      const uint32_t fb = smem_addr(&sh.full_bar[it]);
      mbar_expect_tx(fb, (uint32_t)(kStTileBytes + 2 * ncoef * 4));
      tma_load_2d(sbase + (uint32_t)(it * kStStageBytes), &PP->tmC, c0, r0, fb);
    }
  }
  pdl_wait();
  const bool skip = (mode != MODE_PLAIN && mode != MODE_EVAL && st->done) ||
                    (COL && mode == MODE_TRIAL && !st->nr_ok);
  const PassIo io = pass_io(P, COL, mode, st->cur_f, st->cur_g);
  if (skip) {
    // nothing to do: complete the prefetched stages and let them land
    if (warp == 8) {
      st_produce<COL>(PP, g, io, sh, sbase, t0, t0 + npre, 0, npre);
      if (lane == 0)
        for (int it = 0; it < npre; ++it) mbar_wait(smem_addr(&sh.full_bar[it]), 0, kStWait);
    }
    return;
  }
  if (warp == 8) {
    if (!st_produce<COL>(PP, g, io, sh, sbase, t0, t1, 0, npre) && lane == 0) {
      atomicAdd(&st->numeric, 1);
      sh.err = 1;
    }
    pdl_trigger();
    st_drain(sh, (int)(t1 - t0));
    return;
  }
  st_consume<COL>(P, g, io, sh, st_smem, t0, t1, 0, false);
}

// ---------------------------------------------------------------------------
// Cooperative Sinkhorn loop.
// ---------------------------------------------------------------------------
// Grid-wide barrier (all CTAs co-resident: cooperative launch).  bar[0]
// counts arrivals, bar[1] is the generation; the wait is bounded.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Two levels: CTAs arrive on the counter of their group of 32 (bar[2 + group]),
// the last of a group on the root counter bar[0]; the last root arrival (the
// releaser, run by warp 0 of its CTA) calls on_release() and advances the
// generation bar[1] by 4, its low two bits carrying the code on_release
// returned.  Returns that code to every thread of every CTA, or -1 after a
// wait that gave up.
template <class F>
__device__ int grid_sync(unsigned* bar, unsigned long long wait_ns, StShared& sh, F on_release) {
  __syncthreads();
  const int lane = threadIdx.x & 31;
  if ((threadIdx.x >> 5) == 0) {
    unsigned gen = 0, rel = 0;
    if (lane == 0) {
      gen = ld_acquire(&bar[1]);
      const unsigned grp = blockIdx.x >> 5;
      const unsigned gsz = min(32u, gridDim.x - grp * 32u);
      const unsigned ngrp = (gridDim.x + 31u) >> 5;
      if (arrive_count(&bar[2 + grp]) == gsz - 1) {
        bar[2 + grp] = 0u;
        if (arrive_count(&bar[0]) == ngrp - 1) rel = 1;
      }
    }
    rel = __shfl_sync(0xffffffffu, rel, 0);
    gen = __shfl_sync(0xffffffffu, gen, 0);
    int code = 0;
    if (rel) {
      code = on_release();   // warp-collective
      if (lane == 0) {
        bar[0] = 0u;
        st_release(&bar[1], (gen & ~3u) + 4u + (unsigned)code);
      }
    } else if (lane == 0) {
      unsigned long long t0;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      unsigned now;
      while ((now = ld_acquire(&bar[1])) == gen) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > wait_ns) break;
        __nanosleep(32);
      }
      code = now == gen ? -1 : (int)(now & 3u);
    }
    if (lane == 0) sh.done = code;
  }
  __syncthreads();
  return sh.done;
}

// Sinkhorn iterations (row half-step, then column half-step with the L1 test
// of Algorithm 4.1) until the test passes, max_iter is reached or max_body
// iterations ran in this launch.
__global__ void __launch_bounds__(kStThreads, 2)
    sk_coop_kernel(const Prob* __restrict__ PP, int max_body) {
  const Prob& P = *PP;
  State* st = P.st;
  extern __shared__ __align__(1024) unsigned char st_smem[];
  __shared__ StShared sh;
  const StGeom g(P.n, P.m, (int)gridDim.x);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sbase = smem_addr(st_smem);
  const long long t0 = g.first(blockIdx.x), t1 = g.first(blockIdx.x + 1);
  const int chunk = (int)(t1 - t0);
  st_init_shared(sh);
  // every CTA reads the state before the first barrier's releaser writes it
  if (st->done) return;
  const int cf = st->cur_f;
  int cg = st->cur_g;
  int iter = st->iter;
  const int max_iter = st->max_iter;
  const double tol = st->tol;
  (void)warp;
  unsigned* bar = P.gbar;
  int it = 0;
  int npre = 0;            // tiles of the coming phase whose cost copies are in flight
  bool pre_col = false;    // ... and that phase's direction
  int code = 0;
  int body = 0;
  for (; body < max_body; ++body) {
    // ---- row half-step: f <- g^{C,eps} (Eq. foc_f) ----
    {
      const PassIo io = pass_io(P, false, MODE_SK_ROW, cf, cg);
      if (warp == 8) {
        bool okp = st_produce<false>(PP, g, io, sh, sbase, t0, t1, it, npre);
        npre = 0;
        if (okp) {
          const int want = (int)min((long long)kStStages, t1 - t0);
          pre_col = true;
          npre = st_prefetch<true>(PP, g, sh, sbase, t0, want, it + chunk);
          okp = npre == want;
        }
        if (!okp) sh.err = 1;
      } else {
        st_consume<false>(P, g, io, sh, st_smem, t0, t1, it, true);
      }
      it += chunk;
      // the releaser takes the row sums (the row step of the mode)
      code = grid_sync(bar, P.wait_ns, sh, [&]() -> int {
        double tot[3];
        warp0_grid_sum3(P.sk_acc_row, g.ntr, tot);
        if ((threadIdx.x & 31) == 0) {
          st->l1_row = tot[0];
          st->sum_wL = tot[1];
          st->sum_wout = tot[2];
          st->sum_af = tot[2];
        }
        return 0;
      });
      if (code < 0 || sh.err) break;
    }
    // ---- column half-step: g <- f^{C,eps} (Eq. foc_g) and the L1 test ----
    {
      const PassIo io = pass_io(P, true, MODE_SK_COL, cf, cg);
      if (warp == 8) {
        bool okp = st_produce<true>(PP, g, io, sh, sbase, t0, t1, it, npre);
        npre = 0;
        if (okp) {
          const int want = (int)min((long long)kStStages, t1 - t0);
          pre_col = false;
          npre = st_prefetch<false>(PP, g, sh, sbase, t0, want, it + chunk);
          okp = npre == want;
        }
        if (!okp) sh.err = 1;
      } else {
        st_consume<true>(P, g, io, sh, st_smem, t0, t1, it, true);
      }
      it += chunk;
      ++iter;
      // the releaser takes the decision of Algorithm 4.1 (L1 test) for all
      code = grid_sync(bar, P.wait_ns, sh, [&]() -> int {
        double tot[3];
        warp0_grid_sum3(P.sk_acc_col, g.ntc, tot);
        int done = 0;
        if ((threadIdx.x & 31) == 0) {
          const int numeric = *(volatile int*)&st->numeric;
          if (numeric > 0) done = 3;
          else done = stop_code(st, tot[0], iter, tol, max_iter, P.stall_window);
          st->l1_col = tot[0];
          st->qsemi = st->sum_af + tot[2];   // Q_semi(f_k) = <f_k, a> + <f_k^{C,eps}, b>
          st->sum_wL = tot[1];
          st->sum_wout = tot[2];
          st->iter = iter;
          trace_test(P, st, iter, tot[0], st->qsemi);
          if (done) st->done = done;
          else st->cur_g = io.dst_g;
        }
        return __shfl_sync(0xffffffffu, done, 0);
      });
      if (code != 0 || sh.err) break;
      cg = io.dst_g;
    }
  }
  // a barrier wait or a pipeline wait of this CTA that gave up: the loop
  // stops with the timeout state (the host reports EOT_ETIMEDOUT)
  const bool failed = code < 0 || sh.err;
  if (failed) {
    if (tid == 0) st->done = 5;
  } else if (code == 0 && body >= max_body && blockIdx.x == 0 && tid == 0) {
    st->done = 4;   // iteration cap of this launch
  }
  if (warp == 8) {
    // the row tiles prefetched for an iteration that does not run: complete
    // their stages (any coefficients of the right length) and let them land
    if (npre > 0) {
      if (pre_col) {
        const PassIo io = pass_io(P, true, MODE_SK_COL, cf, cg);
        st_produce<true>(PP, g, io, sh, sbase, t0, t0 + npre, it, npre);
      } else {
        const PassIo io = pass_io(P, false, MODE_SK_ROW, cf, cg);
        st_produce<false>(PP, g, io, sh, sbase, t0, t0 + npre, it, npre);
      }
    }
    st_drain(sh, it + npre);
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
void init_stream_attributes() {
  cudaFuncSetAttribute(stream_pass_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kStSmem);
  cudaFuncSetAttribute(stream_pass_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kStSmem);
  cudaFuncSetAttribute(sk_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStSmem);
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
  int c = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, sk_coop_kernel, kStThreads, kStSmem) !=
      cudaSuccess)
    c = 0;
  cudaGetLastError();
  return min(a, min(b, c));
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

// Launched with programmatic stream serialization: the kernel starts while
// the preceding kernel finishes and waits for it (griddepcontrol.wait) before
// reading anything that kernel may write.
cudaError_t launch_stream_pass(const Prob* dP, const Prob& hP, bool col, int mode,
                               cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(col ? hP.sk_gcol : hP.sk_grow));
  cfg.blockDim = dim3(kStThreads);
  cfg.dynamicSmemBytes = kStSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return col ? cudaLaunchKernelEx(&cfg, stream_pass_kernel<true>, dP, mode)
             : cudaLaunchKernelEx(&cfg, stream_pass_kernel<false>, dP, mode);
}

}  // namespace eotk

namespace eotk {

// Cooperative launch of the Sinkhorn loop (grid = the stream passes' grid,
// which one wave holds).  The grid barrier counter is reset first.
cudaError_t launch_sk_coop(const Prob* dP, const Prob& hP, int max_body, cudaStream_t s) {
  // counters (root and groups) start at zero; the generation carries over
  cudaError_t e = cudaMemsetAsync(hP.gbar, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(hP.gbar + 2, 0, 32 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)hP.sk_gcol);
  cfg.blockDim = dim3(kStThreads);
  cfg.dynamicSmemBytes = kStSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sk_coop_kernel, dP, max_body);
}

EOT_DEBUG_UNIT(stream)

}  // namespace eotk
