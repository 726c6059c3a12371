// Log-sum-exp half-steps with the squared-Euclidean cost formed on the fly on
// the tensor cores (EOT_PREC_SPLIT_TC): the Sinkhorn updates of
// Eq. SK_iterations (Eq. foc_f, Eq. foc_g) without a stored cost matrix.
//
//   C_ij = |x_i|^2 + |y_j|^2 - 2 G_ij,   G = X Y^T  (d <= 64, zero padded)
//
// G is a dense contraction: tiles of 128 output-side points x 128
// reduction-side points x 64 coordinates run as tcgen05 MMAs (kind::tf32,
// M = N = 128, K = 8) with every operand split into TF32 high + low parts and
// the three products x_h y_h, x_h y_l, x_l y_h accumulated in float32 in TMEM
// (the accuracy of a float32 dot product).  Each side's potential enters as
// P = k2 (p - |pt|^2) (log2 units) split into a part on the 2^-q grid and a
// float remainder, the same split for both sides, so the exponent
//     y_ij = (2 k2 G_ij + (P_hi,i + P_hi,j)) + (P_lo,i + P_lo,j)
// has an exact grid sum, one rounding relative to the (small) result and a
// small correction; the reduction side's weight multiplies the exponential.
// Both half-steps therefore see bit for bit the same cost: the column pass
// issues its products in the mirror order of the row pass (x_h y_l before
// x_l y_h), every y_ij is a symmetric function of the two sides, and the
// Sinkhorn iteration has a fixed point to converge to, with the marginal test
// met against the kernel's own cost (which differs from the exact cost by the
// float32 error of the dot products).
//
// CTA (one per SM, persistent over a stream-K chunk of (output tile,
// reduction tile) pairs, output-tile-major):
//   warps 0-7  epilogue: read the accumulator from TMEM (warp w reads lanes
//              32 (w % 4) .. +31 = output points, columns 64 (w / 4) .. +63),
//              form the exponents, keep a running log-sum-exp per point;
//   warp 8     producer: TMA copies (128-byte swizzle) of the output tile
//              (once per piece) and of the reduction tiles (2-stage ring),
//              plus the reduction side's W values;
//   warp 9     MMA issuer and TMEM owner (two 128-column accumulators, so
//              the products of tile t + 1 overlap the epilogue of tile t).
// A piece of an output tile ends with the partial (reference, sum) states of
// its points; the last contributor of a tile merges them and finishes it
// (as in the stored-cost stream passes).  Every wait is bounded.
#include "eot_device.cuh"
#include "eot_internal.h"
#include "pass_common.cuh"
#include "reduce.cuh"
#include "stream_common.cuh"
#include "tc.cuh"

namespace eotk {

constexpr int kGT = 128;                     // points per tile (both sides)
constexpr int kGBox = kGT * 128;             // one TMA box: 128 points x 32 floats (16 KB)
constexpr int kGPart = 2 * kGBox;            // hi or lo part of a tile, both 32-float halves
constexpr int kGStages = 2;
constexpr int kGStageBytes = 2 * kGPart + 2048;        // R hi, R lo, P hi / P lo / w (128 each)
constexpr int kGStageOff = 2 * kGPart;                 // after the output tile (hi, lo)
constexpr int kGSmem = kGStageOff + kGStages * kGStageBytes + 1024;   // + alignment slack
constexpr int kGThreads = 320;
constexpr uint32_t kGTmemCols = 256;
constexpr int kGWait = 1 << 22;
constexpr int kGPend = 8;

struct GmShared {
  uint64_t r_full[kGStages], r_empty[kGStages];
  uint64_t a_full, a_empty;
  uint64_t acc_full[2], acc_empty[2];
  uint32_t tmem;
  float2 hv[2][kGT];      // the two column halves' states per output point
  float mr[8][kGT];
  double ms[8][kGT];
  double red[24];
  unsigned flag;
  int err;
  int pend[kGPend];
  int npend;
};

// Geometry: output side O (points of the potential being updated), reduction
// side R; tile pair t = (t / tR, t % tR).
struct GmGeom {
  int nO, nR, tO, tR, G;
  long long T;
  __device__ GmGeom(int nO_, int nR_, int G_) : nO(nO_), nR(nR_), G(G_) {
    tO = (nO + kGT - 1) / kGT;
    tR = (nR + kGT - 1) / kGT;
    T = (long long)tO * tR;
  }
  __device__ long long first(int k) const { return T * k / G; }
  __device__ void contributors(int b, int& kf, int& nc) const {
    kf = st_owner((long long)b * tR, T, G);
    nc = st_owner((long long)(b + 1) * tR - 1, T, G) - kf + 1;
  }
};

// Finish output tile b from its contributors' partials (256 epilogue threads).
template <bool COL>
__device__ void gm_finish_block(const Prob& P, const GmGeom& g, const PassIo& io, GmShared& sh,
                                int b) {
  State* st = P.st;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int slots = COL ? P.gm_slots_col : P.gm_slots_row;
  const float2* part = COL ? P.gm_part_col : P.gm_part_row;
  unsigned* cnt = COL ? P.gm_cnt_col : P.gm_cnt_row;
  double* bacc = COL ? P.gm_acc_col : P.gm_acc_row;
  const int mode = io.mode;
  int kf, nc;
  g.contributors(b, kf, nc);
  const int c = tid % kGT, h = tid / kGT;   // two groups of 128
  float Rg = -INFINITY;
  double Sg = 0.0;
  if (b * kGT + c < g.nO)
    merge_segments(part + (size_t)b * slots * kGT, nc, kGT, c, h, 2, Rg, Sg);
  sh.mr[h][c] = Rg;
  sh.ms[h][c] = Sg;
  cons_sync();
  const int idx = b * kGT + tid;
  float R = -INFINITY;
  double Sd = 0.0;
  if (tid < kGT) {
    R = sh.mr[0][tid];
    Sd = sh.ms[0][tid];
    merge_dd(R, Sd, sh.mr[1][tid], sh.ms[1][tid]);
  }
  if (tid == 0) cnt[b] = 0u;
  double accv[3] = {0.0, 0.0, 0.0};
  if (tid < kGT && idx < g.nO) {
    double* out;
    Split so;
    if (mode == MODE_PLAIN) {
      out = P.out_plain;
      so = Split{nullptr, nullptr, nullptr, nullptr, nullptr};
    } else if (mode == MODE_EVAL) {
      out = nullptr;
      so = Split{nullptr, nullptr, nullptr, nullptr, nullptr};
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
  cons_sum3(accv, sh.red, kGT);
  if (tid == 0) {
    double* ab = bacc + b * 4;
    ab[0] = accv[0];
    ab[1] = accv[1];
    ab[2] = accv[2];
    sh.flag = (arrive_count(&P.gcnt[COL ? 2 : 3]) == (unsigned)(g.tO - 1)) ? 1u : 0u;
  }
  cons_sync();
  if (!sh.flag) return;
  if (warp == 0) {
    double tot[3];
    warp0_grid_sum3(bacc, g.tO, tot);
    if (tid == 0) {
      P.gcnt[COL ? 2 : 3] = 0u;
      if (COL) final_step(P, mode, tot, io.dst_g);
      else if (mode == MODE_EVAL) st->l1_row = tot[0];
      else final_step(P, mode == MODE_PLAIN ? MODE_PLAIN : MODE_SK_ROW, tot, io.cf);
    }
  }
}

template <bool COL>
__global__ void __launch_bounds__(kGThreads, 1)
    gram_pass_kernel(const Prob* __restrict__ PP, int mode) {
  const Prob& P = *PP;
  State* st = P.st;
  extern __shared__ unsigned char gm_raw[];
  __shared__ GmShared sh;
  const uint32_t raw = smem_addr(gm_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;   // 128-byte swizzle: 1024-byte aligned tiles
  const unsigned char* sbase = gm_raw + (base - raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const GmGeom g(COL ? P.m : P.n, COL ? P.n : P.m, (int)gridDim.x);
  const long long t0 = g.first(blockIdx.x), t1 = g.first(blockIdx.x + 1);
  const CUtensorMap* mapOh = COL ? &PP->tmYh : &PP->tmXh;
  const CUtensorMap* mapOl = COL ? &PP->tmYl : &PP->tmXl;
  const CUtensorMap* mapRh = COL ? &PP->tmXh : &PP->tmYh;
  const CUtensorMap* mapRl = COL ? &PP->tmXl : &PP->tmYl;

  if (tid == 0) {
    for (int s = 0; s < kGStages; ++s) {
      mbar_init(smem_addr(&sh.r_full[s]), 1);
      mbar_init(smem_addr(&sh.r_empty[s]), 1 + 8);   // the MMAs' commit + 8 epilogue warps
    }
    mbar_init(smem_addr(&sh.a_full), 1);
    mbar_init(smem_addr(&sh.a_empty), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_addr(&sh.acc_full[b]), 1);
      mbar_init(smem_addr(&sh.acc_empty[b]), 8);
    }
    sh.err = 0;
    sh.npend = 0;
    mbar_init_fence();
  }
  if (warp == 9) tmem_alloc(smem_addr(&sh.tmem), kGTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;

  pdl_wait();
  const bool skip = (mode != MODE_PLAIN && mode != MODE_EVAL && st->done);
  const PassIo io = pass_io(P, COL, mode, st->cur_f, st->cur_g);

  if (!skip) {
    if (warp == 8) {
      // ---------------- producer ----------------
      if (lane == 0) {
        int it = 0, piece = 0, cur = -1;
        bool ok = true;
        for (long long t = t0; t < t1 && ok; ++t, ++it) {
          const int ob = (int)(t / g.tR), rb = (int)(t - (long long)ob * g.tR);
          if (ob != cur) {
            if (piece > 0 && !mbar_wait(smem_addr(&sh.a_empty), (piece - 1) & 1, kGWait)) {
              ok = false;
              break;
            }
            const uint32_t fa = smem_addr(&sh.a_full);
            mbar_expect_tx(fa, 2u * kGPart);
            for (int part = 0; part < 2; ++part)
              for (int half = 0; half < 2; ++half)
                tma_load_2d(base + part * kGPart + half * kGBox, part ? mapOl : mapOh,
                               half * 32, ob * kGT, fa);
            cur = ob;
            ++piece;
          }
          const int s = it % kGStages;
          if (it >= kGStages &&
              !mbar_wait(smem_addr(&sh.r_empty[s]), ((it / kGStages) - 1) & 1, kGWait)) {
            ok = false;
            break;
          }
          const uint32_t fr = smem_addr(&sh.r_full[s]);
          const uint32_t dst = base + kGStageOff + (uint32_t)(s * kGStageBytes);
          mbar_expect_tx(fr, 2u * kGPart + 3u * kGT * 4u);
          for (int part = 0; part < 2; ++part)
            for (int half = 0; half < 2; ++half)
              tma_load_2d(dst + part * kGPart + half * kGBox, part ? mapRl : mapRh, half * 32,
                             rb * kGT, fr);
          // grid part, remainder and weight of the 128 reduction points (the
          // split arrays are padded to a multiple of 128)
          bulk_load(dst + 2 * kGPart, io.red.K + rb * kGT, kGT * 4u, fr);
          bulk_load(dst + 2 * kGPart + kGT * 4, io.red.KL + rb * kGT, kGT * 4u, fr);
          bulk_load(dst + 2 * kGPart + 2 * kGT * 4, io.red.A + rb * kGT, kGT * 4u, fr);
        }
        if (!ok) {
          atomicAdd(&st->numeric, 1);
          sh.err = 1;
        }
      }
    } else if (warp == 9) {
      // ---------------- MMA issuer ----------------
      if (lane == 0) {
        constexpr uint32_t idesc = idesc_tf32(kGT, kGT);
        int it = 0, piece = 0, cur = -1;
        bool ok = true;
        for (long long t = t0; t < t1 && ok; ++t, ++it) {
          const int ob = (int)(t / g.tR);
          if (ob != cur) {
            if (!mbar_wait(smem_addr(&sh.a_full), piece & 1, kGWait)) { ok = false; break; }
            cur = ob;
            ++piece;
          }
          const int s = it % kGStages, b = it & 1;
          if (!mbar_wait(smem_addr(&sh.r_full[s]), (it / kGStages) & 1, kGWait)) { ok = false; break; }
          if (it >= 2 && !mbar_wait(smem_addr(&sh.acc_empty[b]), ((it >> 1) - 1) & 1, kGWait)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(b * kGT);
          const uint32_t ah = base, al = base + kGPart;
          const uint32_t rh = base + kGStageOff + (uint32_t)(s * kGStageBytes), rl = rh + kGPart;
          // row pass (A = X): x_h y_h, x_h y_l, x_l y_h per k-step; the column
          // pass (A = Y) issues the same products in the same order
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint32_t ko = (uint32_t)((k >> 2) * kGBox + (k & 3) * 32);
            mma_tf32(d, sdesc_sw128(ah + ko), sdesc_sw128(rh + ko), idesc, k > 0 ? 1u : 0u);
            if (COL) {
              mma_tf32(d, sdesc_sw128(al + ko), sdesc_sw128(rh + ko), idesc, 1u);
              mma_tf32(d, sdesc_sw128(ah + ko), sdesc_sw128(rl + ko), idesc, 1u);
            } else {
              mma_tf32(d, sdesc_sw128(ah + ko), sdesc_sw128(rl + ko), idesc, 1u);
              mma_tf32(d, sdesc_sw128(al + ko), sdesc_sw128(rh + ko), idesc, 1u);
            }
          }
          mma_commit(smem_addr(&sh.acc_full[b]));
          mma_commit(smem_addr(&sh.r_empty[s]));
          // last tile of this piece: the output tile may be replaced
          const bool piece_end = (t + 1 == t1) || ((int)((t + 1) / g.tR) != ob);
          if (piece_end) mma_commit(smem_addr(&sh.a_empty));
        }
        if (!ok) {
          atomicAdd(&st->numeric, 1);
          sh.err = 1;
        }
        // the products of the last tile have completed before TMEM is released
        if (it > 0) mbar_wait(smem_addr(&sh.acc_full[(it - 1) & 1]), ((it - 1) >> 1) & 1, kGWait);
      }
    } else {
      // ---------------- epilogue ----------------
      const float k2 = P.k2;
      const float k2x2 = 2.f * k2;
      const int lg = warp & 3, half = warp >> 2;     // TMEM lane group, column half
      const int op = lg * 32 + lane;                 // output point within the tile
      float Ph = 0.f, Pl = 0.f, ref = 0.f, rr = -INFINITY, S = 0.f;
      bool valid = false, werr = false;
      int cur = -1;
      const int slots = COL ? P.gm_slots_col : P.gm_slots_row;
      float2* part = COL ? P.gm_part_col : P.gm_part_row;
      unsigned* cnt = COL ? P.gm_cnt_col : P.gm_cnt_row;

      auto publish = [&](int b) {
        sh.hv[half][op] = f2(ref, S);
        if (cons_sync_or(*(volatile int*)&sh.err)) return;
        if (sh.npend == kGPend) {   // the list is full (tiny problems): finish now
          const int np = sh.npend;
          for (int k = 0; k < np; ++k) gm_finish_block<COL>(P, g, io, sh, sh.pend[k]);
          cons_sync();
          if (tid == 0) sh.npend = 0;
        }
        int kf, nc;
        g.contributors(b, kf, nc);
        if (tid < kGT && b * kGT + tid < g.nO) {
          float R = -INFINITY;
          double Sd = 0.0;
          merge_d(R, Sd, sh.hv[0][tid].x, sh.hv[0][tid].y);
          merge_d(R, Sd, sh.hv[1][tid].x, sh.hv[1][tid].y);
          part[((size_t)b * slots + ((int)blockIdx.x - kf)) * kGT + tid] = f2(R, (float)Sd);
        }
        cons_sync();
        if (tid == 0 && arrive_count(&cnt[b]) == (unsigned)(nc - 1)) sh.pend[sh.npend++] = b;
      };

      int it = 0;
      for (long long t = t0; t < t1; ++t, ++it) {
        const int ob = (int)(t / g.tR), rb = (int)(t - (long long)ob * g.tR);
        if (ob != cur) {
          if (cur >= 0) publish(cur);
          cur = ob;
          const int i = ob * kGT + op;
          valid = i < g.nO;
          Ph = valid ? io.outs.K[i] : 0.f;
          Pl = valid ? io.outs.KL[i] : 0.f;
          ref = 0.f;
          rr = -INFINITY;
          S = 0.f;
        }
        const int s = it % kGStages, b = it & 1;
        if (!werr) {
          // warp-uniform outcome: the TMEM loads below are warp-collective
          const bool okw = mbar_wait(smem_addr(&sh.acc_full[b]), (it >> 1) & 1, kGWait);
          if (__any_sync(0xffffffffu, !okw)) {
            werr = true;
            if (lane == 0) {
              atomicAdd(&st->numeric, 1);
              sh.err = 1;
            }
          }
        }
        if (!werr) {
          tc_fence_after();
          const float* Qh = reinterpret_cast<const float*>(sbase + kGStageOff + s * kGStageBytes +
                                                           2 * kGPart) + half * 64;
          const float* Ql = Qh + kGT;
          const float* Wt = Qh + 2 * kGT;
          const int jrem = g.nR - rb * kGT - half * 64;   // valid columns of this half
          float y[64];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * kGT + half * 64 + q * 16), v);
#pragma unroll
            for (int e = 0; e < 16; e += 4) {
              const float4 h4 = *reinterpret_cast<const float4*>(Qh + q * 16 + e);
              const float4 l4 = *reinterpret_cast<const float4*>(Ql + q * 16 + e);
              // (2 k2 G + (hi_i + hi_j)) + (lo_i + lo_j): the grid sum is exact
              y[q * 16 + e + 0] = __fadd_rn(__fmaf_rn(k2x2, v[e + 0], __fadd_rn(Ph, h4.x)), __fadd_rn(Pl, l4.x));
              y[q * 16 + e + 1] = __fadd_rn(__fmaf_rn(k2x2, v[e + 1], __fadd_rn(Ph, h4.y)), __fadd_rn(Pl, l4.y));
              y[q * 16 + e + 2] = __fadd_rn(__fmaf_rn(k2x2, v[e + 2], __fadd_rn(Ph, h4.z)), __fadd_rn(Pl, l4.z));
              y[q * 16 + e + 3] = __fadd_rn(__fmaf_rn(k2x2, v[e + 3], __fadd_rn(Ph, h4.w)), __fadd_rn(Pl, l4.w));
            }
          }
          // the accumulator has been read: release it to the next products
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive1(smem_addr(&sh.acc_empty[b]));
          if (jrem < 64) {
#pragma unroll
            for (int e = 0; e < 64; ++e) y[e] = e < jrem ? y[e] : -INFINITY;
          }
          float mx = -INFINITY;
#pragma unroll
          for (int e = 0; e < 64; ++e) mx = fmaxf(mx, y[e]);
          rr = fmaxf(rr, mx - ref);
          if (!(fabsf(rr) <= kStWindow && ref == 0.f) && needs_move(rr, ref)) move_ref(rr, ref, S);
          // sum of w_j 2^(y - ref): the weight multiplies the exponential
          float acc = 0.f;
          if (ref == 0.f) {
#pragma unroll
            for (int e = 0; e < 64; ++e) acc = __fmaf_rn(ex2_approx(y[e]), Wt[e], acc);
          } else {
#pragma unroll
            for (int e = 0; e < 64; ++e) acc = __fmaf_rn(ex2_approx(y[e] - ref), Wt[e], acc);
          }
          S += acc;
          // the stage's coefficients have been read: it may be refilled
          __syncwarp();
          if (lane == 0) mbar_arrive1(smem_addr(&sh.r_empty[s]));
        } else {
          __syncwarp();
          if (lane == 0) {
            mbar_arrive1(smem_addr(&sh.acc_empty[b]));
            mbar_arrive1(smem_addr(&sh.r_empty[s]));
          }
        }
      }
      (void)valid;
      pdl_trigger();
      if (cur >= 0) publish(cur);
      if (!cons_sync_or(*(volatile int*)&sh.err)) {
        const int np = sh.npend;
        for (int k = 0; k < np; ++k) gm_finish_block<COL>(P, g, io, sh, sh.pend[k]);
      }
    }
  }
  // TMEM is released after every MMA has completed and every read is done
  tc_fence_before();
  __syncthreads();
  if (warp == 9) {
    tc_fence_after();
    tmem_dealloc(tmem, kGTmemCols);
  }
}

// ---------------------------------------------------------------------------
// Set-up kernels.
// ---------------------------------------------------------------------------
// TF32 high / low parts of n points (row-major, d <= 64) into n x 64 arrays
// (zero padded), and the squared norms in float64; points scaled by `scale`.
__global__ void gram_split_kernel(const float* __restrict__ X, int n, int d, double scale,
                                  float* __restrict__ Xh, float* __restrict__ Xl,
                                  double* __restrict__ nrm, unsigned* __restrict__ bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s2 = 0.0;
    for (int k = 0; k < 64; ++k) {
      float h = 0.f, l = 0.f;
      if (k < d) {
        const double x = (double)X[(size_t)i * d + k] * scale;
        const float xf = (float)x;
        h = to_tf32(xf);
        l = to_tf32(xf - h);
        s2 += (double)xf * (double)xf;
        if (!isfinite(xf)) atomicAdd(bad, 1u);
      }
      Xh[(size_t)i * 64 + k] = h;
      Xl[(size_t)i * 64 + k] = l;
    }
    nrm[i] = s2;
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
void init_gram_attributes() {
  cudaFuncSetAttribute(gram_pass_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kGSmem);
  cudaFuncSetAttribute(gram_pass_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kGSmem);
}

int gram_smem_bytes() { return kGSmem; }

// Grid size and contributor slots of a pass with nO output and nR reduction
// points on `ctas` CTAs.
void gram_plan(int nO, int nR, int ctas, int* grid, int* slots) {
  const long long tO = (nO + kGT - 1) / kGT, tR = (nR + kGT - 1) / kGT;
  const long long T = tO * tR;
  long long G = ctas;
  if (G > T) G = T;
  if (G < 1) G = 1;
  long long mx = 1;
  for (long long b = 0; b < tO; ++b) {
    const long long kf = ((b * tR + 1) * G - 1) / T;
    const long long kl = (((b + 1) * tR) * G - 1) / T;
    if (kl - kf + 1 > mx) mx = kl - kf + 1;
  }
  *grid = (int)G;
  *slots = (int)mx;
}

cudaError_t launch_gram_pass(const Prob* dP, const Prob& hP, bool col, int mode, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(col ? hP.gm_gcol : hP.gm_grow));
  cfg.blockDim = dim3(kGThreads);
  cfg.dynamicSmemBytes = kGSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return col ? cudaLaunchKernelEx(&cfg, gram_pass_kernel<true>, dP, mode)
             : cudaLaunchKernelEx(&cfg, gram_pass_kernel<false>, dP, mode);
}

cudaError_t launch_gram_split(const float* X, int n, int d, double scale, float* Xh, float* Xl,
                              double* nrm, unsigned* bad, cudaStream_t s) {
  const int blocks = (n + 255) / 256;
  gram_split_kernel<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(X, n, d, scale, Xh, Xl, nrm,
                                                                   bad);
  return cudaGetLastError();
}

}  // namespace eotk
