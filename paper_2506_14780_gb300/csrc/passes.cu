// Log-domain Sinkhorn half-steps on a stored float32 cost (paper Eq. foc_f,
// Eq. foc_g, Eq. SK_iterations), with their reductions fused:
//
//   column pass  out_j = s_j - eps * L_j,  L_j = log sum_i exp(x_ij),
//                x_ij  = log a_i + (u_i + s_j - C_ij)/eps
//   row pass     out_i = s_i - eps * L_i,  L_i = log sum_j exp(x_ij),
//                x_ij  = log b_j + (s_i + u_j - C_ij)/eps
//
// s is the current potential on the output side (a shift that keeps x near 0
// at convergence; the result does not depend on it in exact arithmetic) and u
// the potential on the reduction side.  exp(L_j) is the marginal ratio
// (pi^T 1)_j / b_j of pi(u, s), so the same pass yields the marginal error used
// by the stopping test of Algorithm 4.1 (and L1 of a column pass at f_k is
// ||pi^T 1 - b||_1 for pi(f_k, g_k)).
//
// Layout: C row-major n x m.  Column pass: CTA = 128 columns (32 lanes x float4)
// x one stripe of rows, 8 warps interleaved over the stripe's rows, every warp
// load a 512-byte run; the next four rows of a warp are fetched into registers
// while the current four are reduced.  Row pass: CTA = 32 rows (4 per warp) x
// one segment of columns, lanes along the row with float4 loads, the next step
// prefetched the same way.  Partial (reference, sum) states go to a
// [segment][index] buffer; the last CTA to finish an index block (atomic
// arrival counter) merges the segments in parallel and in a fixed order, so
// results are deterministic; the last index block then runs the mode-specific
// grid-wide step.
#include <algorithm>

#include "eot_device.cuh"
#include "eot_internal.h"
#include "reduce.cuh"
#include "pass_common.cuh"

namespace eotk {

// ---------------------------------------------------------------------------
// Column pass.  VEC = 4: m % 4 == 0 (16-byte aligned rows), float4 loads;
// VEC = 1: scalar loads with column bounds checks.
// ---------------------------------------------------------------------------
template <int VEC, bool ACC>
__global__ void __launch_bounds__(kThreads) col_pass_kernel(const Prob* __restrict__ PP, int mode) {
  const Prob& P = *PP;
  State* st = P.st;
  if (mode != MODE_PLAIN && mode != MODE_EVAL && st->done) return;
  const int cf = st->cur_f, cg = st->cur_g;
  // source f, shift g and destination g buffers: a trial pass (Algorithm 4.1,
  // value at f' = f_k + V Delta) reads f' and is shifted by h = f_k^{C,eps}.
  const int src_f = (mode == MODE_TRIAL) ? 1 - cf : cf;
  const int sh_g = (mode == MODE_TRIAL) ? (cg + 1) % 3 : cg;
  const int dst_g = (mode == MODE_EVAL) ? -1 : (mode == MODE_TRIAL ? (cg + 2) % 3 : (cg + 1) % 3);
  if (mode == MODE_TRIAL && !st->nr_ok) return;
  const float* __restrict__ rA = P.rs[src_f].A;
  const float* __restrict__ rAL = P.rs[src_f].AL;
  const float* __restrict__ cK = P.cs[sh_g].K;
  const float* __restrict__ cKL = P.cs[sh_g].KL;

  __shared__ float2 s_part[8][kColTile];
  __shared__ float s_cr[2][kColTile];
  __shared__ double s_cs[2][kColTile];
  __shared__ double s_red[24];
  __shared__ unsigned s_last;

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n = P.n, m = P.m;
  const int cb = blockIdx.x, stripe = blockIdx.y;
  const int j0 = cb * kColTile + lane * 4;
  const int i_beg = stripe * P.rows_per_stripe;
  const int nrows = min(n, i_beg + P.rows_per_stripe) - i_beg;
  const float k2 = P.k2, k2lo = P.k2lo;

  float K[4], cc0[4], cc[4], ref[4], run[4], S[4];
  bool valid[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = j0 + c;
    valid[c] = j < m;
    K[c] = valid[c] ? cK[j] : P.M;
    cc0[c] = valid[c] ? cKL[j] * k2 : 0.f;
    cc[c] = cc0[c];
    ref[c] = 0.f;
    run[c] = -INFINITY;
    S[c] = 0.f;
  }

  if (valid[0]) {
    // rows r = wid + 8 t of the stripe, four at a time, prefetched one step ahead
    float cn[4][4], an[4], aln[4];
    auto fetch = [&](int r0) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + 8 * u;
        if (r < nrows) {
          const int i = i_beg + r;
          const float* crow = P.C + (size_t)i * m + j0;
          if (VEC == 4) {
            const float4 c4 = __ldg(reinterpret_cast<const float4*>(crow));
            cn[u][0] = c4.x; cn[u][1] = c4.y; cn[u][2] = c4.z; cn[u][3] = c4.w;
          } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) cn[u][c] = valid[c] ? __ldg(crow + c) : 0.f;
          }
          an[u] = __ldg(rA + i);
          aln[u] = __ldg(rAL + i);
        }
      }
    };
    fetch(wid);
    for (int r0 = wid; r0 < nrows; r0 += 32) {
      float cv[4][4], av[4], alv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        av[u] = an[u];
        alv[u] = aln[u];
#pragma unroll
        for (int c = 0; c < 4; ++c) cv[u][c] = cn[u][c];
      }
      if (r0 + 32 < nrows) fetch(r0 + 32);
      float t[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool rvalid = r0 + 8 * u < nrows;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          t[u][c] = rvalid ? (ACC ? split_exponent(cv[u][c], K[c], av[u])
                                  : __fadd_rn(split_exponent(cv[u][c], K[c], av[u]), alv[u]))
                           : -INFINITY;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = __fmaf_rn(t[u][c], k2, cc[c]);
        const float mx = fmaxf(fmaxf(y[0], y[1]), fmaxf(y[2], y[3]));
        run[c] = fmaxf(run[c], mx);
        if (run[c] > kRecenter || (run[c] < -kRecenter && run[c] > -INFINITY)) {
          const float d = rintf(run[c]);
          S[c] = scale2(S[c], -d);
          ref[c] += d;
          cc[c] = __fsub_rn(cc0[c], ref[c]);
          run[c] -= d;
#pragma unroll
          for (int u = 0; u < 4; ++u) y[u] = __fmaf_rn(t[u][c], k2, cc[c]);
        }
        if (ACC) {
          // evaluation: the exponent as p + q (ex2_pq), p = t k2 rounded, q its
          // exact rounding error plus the low parts
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float pz = __fmul_rn(t[u][c], k2);   // not contracted with its uses
            const float qz = __fmaf_rn(t[u][c], k2, -pz) +
                             __fmaf_rn(t[u][c], k2lo, __fmaf_rn(alv[u], k2, cc0[c]));
            S[c] += ex2_pq(__fsub_rn(pz, ref[c]), qz);
          }
        } else {
          S[c] += (ex2_approx(y[0]) + ex2_approx(y[1])) + (ex2_approx(y[2]) + ex2_approx(y[3]));
        }
      }
    }
  }
  // intra-CTA combine over the 8 warps (float64 sum at the largest reference)
#pragma unroll
  for (int c = 0; c < 4; ++c) s_part[wid][lane * 4 + c] = make_float2(ref[c], valid[c] ? S[c] : 0.f);
  __syncthreads();
  if (threadIdx.x < kColTile) {
    const int j = cb * kColTile + threadIdx.x;
    float R = -INFINITY;
    double Sd = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const float2 q = s_part[w][threadIdx.x];
      merge_d(R, Sd, q.x, q.y);
    }
    if (j < m && EOT_CHECK(stripe < P.nstripe, 401))
      P.part_col[(size_t)stripe * m + j] = make_float2(R, (float)Sd);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&P.cnt_col[cb], 1u);
    s_last = (prev == (unsigned)(P.nstripe - 1));
  }
  __syncthreads();
  if (!s_last) return;
  // --- this CTA combines column block cb: both halves of the CTA merge half
  //     of the stripes each, then thread c merges the two halves ---
  __threadfence();
  {
    const int c = threadIdx.x & (kColTile - 1), h = threadIdx.x >> 7;
    const int j = cb * kColTile + c;
    float R = -INFINITY;
    double Sd = 0.0;
    if (j < m) merge_segments(P.part_col, P.nstripe, m, j, h, 2, R, Sd);
    s_cr[h][c] = R;
    s_cs[h][c] = Sd;
  }
  __syncthreads();
  double accv[3] = {0.0, 0.0, 0.0};
  if (threadIdx.x < kColTile) {
    const int j = cb * kColTile + threadIdx.x;
    if (j < m) {
      float R = s_cr[0][threadIdx.x];
      double Sd = s_cs[0][threadIdx.x];
      merge_dd(R, Sd, s_cr[1][threadIdx.x], s_cs[1][threadIdx.x]);
      double* out;
      Split so;
      if (mode == MODE_PLAIN) {
        out = P.out_plain;
        so = Split{nullptr, nullptr, nullptr, nullptr};
      } else if (mode == MODE_EVAL) {
        out = nullptr;
        so = Split{nullptr, nullptr, nullptr, nullptr};
      } else {
        out = P.g[dst_g];
        so = P.cs[dst_g];
      }
      finish_index(R, Sd, j, P, P.g[sh_g], P.b, P.logb, out, so, P.Lcol, accv, &st->numeric);
      if (mode == MODE_PLAIN && P.logratio_plain) P.logratio_plain[j] = (double)P.Lcol[j];
    }
  }
  block_sum3(accv, s_red);
  if (threadIdx.x == 0) {
    P.cnt_col[cb] = 0u;
    double* ab = P.acc_col + cb * 4;
    ab[0] = accv[0];
    ab[1] = accv[1];
    ab[2] = accv[2];
    __threadfence();
    const unsigned prev = atomicAdd(&P.gcnt[0], 1u);
    s_last = (prev == (unsigned)(P.ncolblk - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double tot[3];
  grid_sum3(P.acc_col, P.ncolblk, tot, s_red);
  if (threadIdx.x == 0) {
    P.gcnt[0] = 0u;
    final_step(P, mode, tot, dst_g);
  }
}

// ---------------------------------------------------------------------------
// Row pass.
// ---------------------------------------------------------------------------
template <int VEC, bool ACC>
__global__ void __launch_bounds__(kThreads) row_pass_kernel(const Prob* __restrict__ PP, int mode) {
  const Prob& P = *PP;
  State* st = P.st;
  if (mode != MODE_PLAIN && mode != MODE_EVAL && st->done) return;
  const int cf = st->cur_f, cg = st->cur_g;
  const float* __restrict__ cA = P.cs[cg].A;
  const float* __restrict__ cAL = P.cs[cg].AL;
  const float* __restrict__ rK = P.rs[cf].K;
  const float* __restrict__ rKL = P.rs[cf].KL;

  __shared__ float2 s_part[kRowTile];
  __shared__ float s_cr[8][kRowTile];
  __shared__ double s_cs[8][kRowTile];
  __shared__ double s_red[24];
  __shared__ unsigned s_last;

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n = P.n, m = P.m;
  const int rb = blockIdx.x, seg = blockIdx.y;
  const int i0 = rb * kRowTile + wid * kRowsPerWarp;
  const int c_beg = seg * P.cols_per_seg;
  const int c_end = min(m, c_beg + P.cols_per_seg);
  const float k2 = P.k2, k2lo = P.k2lo;

  float K[kRowsPerWarp], cc0[kRowsPerWarp], cc[kRowsPerWarp], ref[kRowsPerWarp],
      run[kRowsPerWarp], S[kRowsPerWarp];
  bool rv[kRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int i = i0 + r;
    rv[r] = i < n;
    K[r] = rv[r] ? rK[i] : P.M;
    cc0[r] = rv[r] ? rKL[i] * k2 : 0.f;
    cc[r] = cc0[r];
    ref[r] = 0.f;
    run[r] = -INFINITY;
    S[r] = 0.f;
  }
  if (rv[0]) {
    float can[4], caln[4], cn[kRowsPerWarp][4];
    auto fetch = [&](int j) {
      if (VEC == 4) {
        const float4 a4 = __ldg(reinterpret_cast<const float4*>(cA + j));
        const float4 l4 = __ldg(reinterpret_cast<const float4*>(cAL + j));
        can[0] = a4.x; can[1] = a4.y; can[2] = a4.z; can[3] = a4.w;
        caln[0] = l4.x; caln[1] = l4.y; caln[2] = l4.z; caln[3] = l4.w;
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const bool v = j + c < c_end;
          can[c] = v ? __ldg(cA + j + c) : 0.f;
          caln[c] = v ? __ldg(cAL + j + c) : 0.f;
        }
      }
#pragma unroll
      for (int r = 0; r < kRowsPerWarp; ++r) {
        if (rv[r]) {
          const float* crow = P.C + (size_t)(i0 + r) * m + j;
          if (VEC == 4) {
            const float4 c4 = __ldg(reinterpret_cast<const float4*>(crow));
            cn[r][0] = c4.x; cn[r][1] = c4.y; cn[r][2] = c4.z; cn[r][3] = c4.w;
          } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) cn[r][c] = (j + c < c_end) ? __ldg(crow + c) : 0.f;
          }
        }
      }
    };
    int j = c_beg + lane * 4;
    if (j < c_end) fetch(j);
    for (; j < c_end; j += 128) {
      float ca[4], cal[4], cv[kRowsPerWarp][4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        ca[c] = can[c];
        cal[c] = caln[c];
      }
#pragma unroll
      for (int r = 0; r < kRowsPerWarp; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cv[r][c] = cn[r][c];
      if (j + 128 < c_end) fetch(j + 128);
      bool cvld[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) cvld[c] = (VEC == 4) || (j + c < c_end);
#pragma unroll
      for (int r = 0; r < kRowsPerWarp; ++r) {
        float t[4], y[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          t[c] = (cvld[c] && rv[r]) ? (ACC ? split_exponent(cv[r][c], K[r], ca[c])
                                           : __fadd_rn(split_exponent(cv[r][c], K[r], ca[c]), cal[c]))
                                    : -INFINITY;
          y[c] = __fmaf_rn(t[c], k2, cc[r]);
        }
        const float mx = fmaxf(fmaxf(y[0], y[1]), fmaxf(y[2], y[3]));
        run[r] = fmaxf(run[r], mx);
        if (run[r] > kRecenter || (run[r] < -kRecenter && run[r] > -INFINITY)) {
          const float d = rintf(run[r]);
          S[r] = scale2(S[r], -d);
          ref[r] += d;
          cc[r] = __fsub_rn(cc0[r], ref[r]);
          run[r] -= d;
#pragma unroll
          for (int c = 0; c < 4; ++c) y[c] = __fmaf_rn(t[c], k2, cc[r]);
        }
        if (ACC) {
          // evaluation: p + q as in the column pass
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float pz = __fmul_rn(t[c], k2);
            const float qz = __fmaf_rn(t[c], k2, -pz) +
                             __fmaf_rn(t[c], k2lo, __fmaf_rn(cal[c], k2, cc0[r]));
            S[r] += ex2_pq(__fsub_rn(pz, ref[r]), qz);
          }
        } else {
          S[r] += (ex2_approx(y[0]) + ex2_approx(y[1])) + (ex2_approx(y[2]) + ex2_approx(y[3]));
        }
      }
    }
  }
  // warp reduction of each row's state
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    float rr = ref[r], ss = S[r];
    const bool uniform = __all_sync(0xffffffffu, rr == __shfl_sync(0xffffffffu, rr, 0));
    if (uniform) {
      ss = warp_sum_f(ss);
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float r2 = __shfl_xor_sync(0xffffffffu, rr, o);
        const float s2 = __shfl_xor_sync(0xffffffffu, ss, o);
        lse2_merge(rr, ss, r2, s2);
      }
    }
    if (lane == 0) s_part[wid * kRowsPerWarp + r] = make_float2(rr, ss);
  }
  __syncthreads();
  if (threadIdx.x < kRowTile) {
    const int i = rb * kRowTile + threadIdx.x;
    if (i < n) P.part_row[(size_t)seg * n + i] = s_part[threadIdx.x];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&P.cnt_row[rb], 1u);
    s_last = (prev == (unsigned)(P.nseg - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  {
    // eight groups of 32 threads merge interleaved segments of the 32 rows
    const int rr = threadIdx.x & (kRowTile - 1), h = threadIdx.x >> 5;
    const int i = rb * kRowTile + rr;
    float R = -INFINITY;
    double Sd = 0.0;
    if (i < n) merge_segments(P.part_row, P.nseg, n, i, h, 8, R, Sd);
    s_cr[h][rr] = R;
    s_cs[h][rr] = Sd;
  }
  __syncthreads();
  double accv[3] = {0.0, 0.0, 0.0};
  if (threadIdx.x < kRowTile) {
    const int i = rb * kRowTile + threadIdx.x;
    if (i < n) {
      float R = s_cr[0][threadIdx.x];
      double Sd = s_cs[0][threadIdx.x];
#pragma unroll
      for (int h = 1; h < 8; ++h) merge_dd(R, Sd, s_cr[h][threadIdx.x], s_cs[h][threadIdx.x]);
      double* out;
      Split so;
      if (mode == MODE_PLAIN) {
        out = P.out_plain;
        so = Split{nullptr, nullptr, nullptr, nullptr};
      } else if (mode == MODE_EVAL) {
        out = nullptr;
        so = Split{nullptr, nullptr, nullptr, nullptr};
      } else {
        out = P.f[cf];
        so = P.rs[cf];
      }
      finish_index(R, Sd, i, P, P.f[cf], P.a, P.loga, out, so, P.Lrow, accv, &st->numeric);
      if (mode == MODE_PLAIN && P.logratio_plain) P.logratio_plain[i] = (double)P.Lrow[i];
    }
  }
  block_sum3(accv, s_red);
  if (threadIdx.x == 0) {
    P.cnt_row[rb] = 0u;
    double* ab = P.acc_row + rb * 4;
    ab[0] = accv[0];
    ab[1] = accv[1];
    ab[2] = accv[2];
    __threadfence();
    const unsigned prev = atomicAdd(&P.gcnt[1], 1u);
    s_last = (prev == (unsigned)(P.nrowblk - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double tot[3];
  grid_sum3(P.acc_row, P.nrowblk, tot, s_red);
  if (threadIdx.x == 0) {
    P.gcnt[1] = 0u;
    if (mode == MODE_EVAL) st->l1_row = tot[0];
    else final_step(P, mode == MODE_PLAIN ? MODE_PLAIN : MODE_SK_ROW, tot, cf);
  }
}

// ---------------------------------------------------------------------------
// Split arrays of a float64 potential (level start, after f' = f + V Delta...).
// ---------------------------------------------------------------------------
__global__ void split_kernel(const Prob* __restrict__ PP, const double* __restrict__ p,
                             const double* __restrict__ logw, int len, Split so) {
  const Prob& P = *PP;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
    const double v = p[i];
    if (so.nrm) {   // on-the-fly cost
      double hi;
      float lo;
      split_grid((double)P.k2 * (v - so.nrm[i]), P.qscale, P.qinv, hi, lo);
      so.A[i] = (float)exp(logw[i]);
      so.AL[i] = 0.f;
      so.K[i] = (float)hi;
      so.KL[i] = lo;
      continue;
    }
    double hi;
    float lo;
    split_grid(v + P.eps * logw[i], P.qscale, P.qinv, hi, lo);
    so.A[i] = (float)(hi + (double)P.M);
    so.AL[i] = lo;
    split_grid(v, P.qscale, P.qinv, hi, lo);
    so.K[i] = (float)((double)P.M - hi);
    so.KL[i] = lo;
  }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers.
// ---------------------------------------------------------------------------
cudaError_t launch_stream_pass(const Prob* dP, const Prob& hP, bool col, int mode,
                               cudaStream_t s);

// The staged stream kernels (stream.cu) take every pass whose cost rows are
// 16-byte aligned; the striped kernels below serve the rest.
static bool stream_ok(const Prob& hP, bool col) {
  return (col ? hP.sk_gcol : hP.sk_grow) > 0 && hP.has_tmC;
}

// The evaluation passes (MODE_EVAL: the verification of a returned pair and
// its scores) run on the striped kernels with the unbiased exponential.
cudaError_t launch_col_pass(const Prob* dP, const Prob& hP, int mode, cudaStream_t s) {
  const bool acc = mode == MODE_EVAL;
  if (!acc && stream_ok(hP, true)) return launch_stream_pass(dP, hP, true, mode, s);
  dim3 grid(hP.ncolblk, hP.nstripe);
  const bool v4 = hP.m % 4 == 0 && (reinterpret_cast<uintptr_t>(hP.C) & 15u) == 0;
  if (v4 && acc) col_pass_kernel<4, true><<<grid, kThreads, 0, s>>>(dP, mode);
  else if (v4) col_pass_kernel<4, false><<<grid, kThreads, 0, s>>>(dP, mode);
  else if (acc) col_pass_kernel<1, true><<<grid, kThreads, 0, s>>>(dP, mode);
  else col_pass_kernel<1, false><<<grid, kThreads, 0, s>>>(dP, mode);
  return cudaGetLastError();
}

cudaError_t launch_row_pass(const Prob* dP, const Prob& hP, int mode, cudaStream_t s) {
  const bool acc = mode == MODE_EVAL;
  if (!acc && stream_ok(hP, false)) return launch_stream_pass(dP, hP, false, mode, s);
  dim3 grid(hP.nrowblk, hP.nseg);
  const bool v4 = hP.m % 4 == 0 && (reinterpret_cast<uintptr_t>(hP.C) & 15u) == 0 &&
                  hP.cols_per_seg % 4 == 0;
  if (v4 && acc) row_pass_kernel<4, true><<<grid, kThreads, 0, s>>>(dP, mode);
  else if (v4) row_pass_kernel<4, false><<<grid, kThreads, 0, s>>>(dP, mode);
  else if (acc) row_pass_kernel<1, true><<<grid, kThreads, 0, s>>>(dP, mode);
  else row_pass_kernel<1, false><<<grid, kThreads, 0, s>>>(dP, mode);
  return cudaGetLastError();
}

cudaError_t launch_split(const Prob* dP, const double* p, const double* logw, int len, Split so,
                         cudaStream_t s) {
  const int blocks = (len + 255) / 256;
  split_kernel<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(dP, p, logw, len, so);
  return cudaGetLastError();
}

}  // namespace eotk

// ===========================================================================
// Float64 passes (EOT_PREC_FP64): the same half-steps with float64 costs,
// exponentials and sums, for small problems and tight tolerances.  Column
// pass: one thread per column, 128 columns per CTA, row stripes; row pass: one
// warp per row, column segments.  The partial states are (max, sum) pairs in
// natural-log units, merged in fixed order by the last-arriving CTA.
// ===========================================================================
namespace eotk {

__device__ __forceinline__ void lse64_push(double& mx, double& S, double x) {
  if (x <= mx) {
    S += exp(x - mx);
  } else {
    S = S * exp(mx - x) + 1.0;
    mx = x;
  }
}

__device__ __forceinline__ void lse64_merge(double& mx, double& S, double m2, double S2) {
  if (!(S2 > 0.0)) return;
  if (!(S > 0.0)) {
    mx = m2;
    S = S2;
    return;
  }
  if (m2 <= mx) S += S2 * exp(m2 - mx);
  else {
    S = S * exp(mx - m2) + S2;
    mx = m2;
  }
}

// Finish one index in float64: new potential, its eps-shifted copy, the float
// log-ratio, the scalar contributions.
__device__ __forceinline__ void finish64(double mx, double S, int idx, const Prob& P,
                                         const double* __restrict__ shift,
                                         const double* __restrict__ w,
                                         const double* __restrict__ logw,
                                         double* __restrict__ out, double* __restrict__ outA,
                                         float* __restrict__ Lout, double acc[3], int* numeric,
                                         double* Lfull) {
  double L = mx + log(S);
  const double sh = shift[idx];
  double o = sh - P.eps * L;
  if (!isfinite(o) || !(S > 0.0)) {
    atomicAdd(numeric, 1);
    o = sh;
    L = 0.0;
  }
  if (out) out[idx] = o;
  if (outA) outA[idx] = o + P.eps * logw[idx];
  if (Lout) Lout[idx] = (float)L;
  if (Lfull) *Lfull = L;
  const double wi = w[idx];
  acc[0] = wi * fabs(expm1(L));
  acc[1] = wi * L;
  acc[2] = wi * o;
}

// mode: PLAIN, SK_COL, G_INIT, EVAL, TRIAL, or S4 (with W accumulation; the
// whole column in one stripe).
__global__ void __launch_bounds__(128) col64_kernel(const Prob* __restrict__ PP, int mode,
                                                    AccArgs acc_args) {
  const Prob& P = *PP;
  State* st = P.st;
  if (mode != MODE_PLAIN && mode != MODE_EVAL && st->done) return;
  const bool s4 = mode == MODE_S4;
  const int cf = st->cur_f, cg = st->cur_g;
  const int src_f = (mode == MODE_TRIAL) ? 1 - cf : cf;
  const int sh_g = (mode == MODE_TRIAL) ? (cg + 1) % 3 : cg;
  const int dst_g = (mode == MODE_EVAL) ? -1 : (mode == MODE_TRIAL ? (cg + 2) % 3 : (cg + 1) % 3);
  if (mode == MODE_TRIAL && !st->nr_ok) return;
  const double* __restrict__ fA = P.fA64[src_f];
  __shared__ double s_red[24];
  __shared__ unsigned s_last;
  __shared__ float sW[128 * (kMaxK + 1)];
  __shared__ float sD[128], sB[128];
  const int tid = threadIdx.x;
  const int n = P.n, m = P.m;
  const int cb = blockIdx.x, stripe = blockIdx.y;
  const int j = cb * 128 + tid;
  const bool jv = j < m;
  const int i_beg = s4 ? 0 : stripe * P.rows_per_stripe;
  const int i_end = s4 ? n : min(n, i_beg + P.rows_per_stripe);
  const double inv_eps = 1.0 / P.eps;
  const int kk = s4 ? P.ell : 0;
  double mx = -INFINITY, S = 0.0;
  double w[kMaxK];
  for (int k = 0; k < kk; ++k) w[k] = 0.0;
  if (jv) {
    const double s = P.g[sh_g][j];
    for (int i = i_beg; i < i_end; ++i) {
      const double x = (fA[i] + s - P.C64[(size_t)i * m + j]) * inv_eps;
      if (!s4) {
        lse64_push(mx, S, x);
      } else {
        if (x > mx) {
          const double sc = (S > 0.0) ? exp(mx - x) : 0.0;
          S *= sc;
          for (int k = 0; k < kk; ++k) w[k] *= sc;
          mx = x;
        }
        const double e = exp(x - mx);
        S += e;
        const float* Vi = P.V + (size_t)i * kk;
        for (int k = 0; k < kk; ++k) w[k] += e * (double)Vi[k];
      }
    }
  }
  double accv[3] = {0.0, 0.0, 0.0};
  if (s4) {
    // single stripe: finish directly
    sD[tid] = 0.f;
    sB[tid] = 0.f;
    for (int k = 0; k < kk; ++k) sW[tid * (kMaxK + 1) + k] = 0.f;
    if (jv) {
      double L;
      finish64(mx, S, j, P, P.g[sh_g], P.b, P.logb, P.g[dst_g], P.gA64[dst_g], P.Lcol, accv,
               &st->numeric, &L);
      const double sc = P.b[j] / S;   // b_j * softmax normalisation
      for (int k = 0; k < kk; ++k) {
        const float wv = (float)(w[k] * sc);
        P.W[(size_t)j * kk + k] = wv;
        sW[tid * (kMaxK + 1) + k] = wv;
      }
      const double dj = -expm1(L);
      acc_args.dw[j] = dj;
      sD[tid] = (float)dj;
      sB[tid] = (float)(1.0 / P.b[j]);
    }
    __syncthreads();
    double* dstp = acc_args.wtw_part + (size_t)cb * (kk * kk + kk);
    for (int e = tid; e < kk * kk + kk; e += 128) {
      float s = 0.f;
      if (e < kk * kk) {
        const int r = e / kk, q2 = e - r * kk;
        for (int q = 0; q < 128; ++q)
          s = __fmaf_rn(sW[q * (kMaxK + 1) + r] * sB[q], sW[q * (kMaxK + 1) + q2], s);
      } else {
        const int r = e - kk * kk;
        for (int q = 0; q < 128; ++q) s = __fmaf_rn(sD[q], sW[q * (kMaxK + 1) + r], s);
      }
      dstp[e] = (double)s;
    }
    block_sum3(accv, s_red);
    if (tid == 0) {
      double* ab = acc_args.blkacc + cb * 4;
      ab[0] = accv[0];
      ab[1] = accv[1];
      ab[2] = accv[2];
      __threadfence();
      const unsigned prev = atomicAdd(acc_args.gcnt, 1u);
      s_last = (prev == (unsigned)(acc_args.nblk - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double tot[3];
    grid_sum3(acc_args.blkacc, acc_args.nblk, tot, s_red);
    if (tid == 0) {
      *acc_args.gcnt = 0u;
      st->l1_col = tot[0];
      st->sum_wL = tot[1];
      st->qsemi = st->sum_af + tot[2];
      st->iter += 1;
      trace_test(P, st, st->iter, tot[0], st->qsemi);
      st->nr_ok = 0;
      if (st->numeric > 0) st->done = 3;
      else st->done = stop_code(st, tot[0], st->iter, st->tol, st->max_iter, P.stall_window);
    }
    return;
  }
  if (jv) P.part64_col[(size_t)stripe * m + j] = make_double2(mx, S);
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned prev = atomicAdd(&P.cnt_col[cb], 1u);
    s_last = (prev == (unsigned)(P.nstripe - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (jv) {
    double M = -INFINITY, Sd = 0.0;
    for (int s2 = 0; s2 < P.nstripe; ++s2) {
      const double2 q = __ldcg(&P.part64_col[(size_t)s2 * m + j]);
      lse64_merge(M, Sd, q.x, q.y);
    }
    double* out = (mode == MODE_PLAIN) ? P.out_plain : (mode == MODE_EVAL ? nullptr : P.g[dst_g]);
    double* outA = (mode == MODE_PLAIN || mode == MODE_EVAL) ? nullptr : P.gA64[dst_g];
    double L;
    finish64(M, Sd, j, P, P.g[sh_g], P.b, P.logb, out, outA, P.Lcol, accv, &st->numeric, &L);
    if (mode == MODE_PLAIN && P.logratio_plain) P.logratio_plain[j] = L;
  }
  __syncthreads();
  block_sum3(accv, s_red);
  if (tid == 0) {
    P.cnt_col[cb] = 0u;
    double* ab = P.acc_col + cb * 4;
    ab[0] = accv[0];
    ab[1] = accv[1];
    ab[2] = accv[2];
    __threadfence();
    const unsigned prev = atomicAdd(&P.gcnt[0], 1u);
    s_last = (prev == (unsigned)(P.ncolblk64 - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double tot[3];
  grid_sum3(P.acc_col, P.ncolblk64, tot, s_red);
  if (tid == 0) {
    P.gcnt[0] = 0u;
    final_step(P, mode, tot, dst_g);
  }
}

__global__ void __launch_bounds__(256) row64_kernel(const Prob* __restrict__ PP, int mode) {
  const Prob& P = *PP;
  State* st = P.st;
  if (mode != MODE_PLAIN && mode != MODE_EVAL && st->done) return;
  const int cf = st->cur_f, cg = st->cur_g;
  const double* __restrict__ gA = P.gA64[cg];
  __shared__ double s_red[24];
  __shared__ double2 s_p[8];
  __shared__ unsigned s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n = P.n, m = P.m;
  const int rb = blockIdx.x, seg = blockIdx.y;
  const int i = rb * 8 + wid;
  const int c_beg = seg * P.cols_per_seg;
  const int c_end = min(m, c_beg + P.cols_per_seg);
  const double inv_eps = 1.0 / P.eps;
  double mx = -INFINITY, S = 0.0;
  if (i < n) {
    const double s = P.f[cf][i];
    for (int j = c_beg + lane; j < c_end; j += 32) {
      const double x = (s + gA[j] - P.C64[(size_t)i * m + j]) * inv_eps;
      lse64_push(mx, S, x);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double m2 = __shfl_xor_sync(0xffffffffu, mx, o);
    const double s2 = __shfl_xor_sync(0xffffffffu, S, o);
    lse64_merge(mx, S, m2, s2);
  }
  if (lane == 0) s_p[wid] = make_double2(mx, S);
  __syncthreads();
  if (threadIdx.x < 8) {
    const int ii = rb * 8 + threadIdx.x;
    if (ii < n) P.part64_row[(size_t)seg * n + ii] = s_p[threadIdx.x];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&P.cnt_row[rb], 1u);
    s_last = (prev == (unsigned)(P.nseg - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double accv[3] = {0.0, 0.0, 0.0};
  if (threadIdx.x < 8) {
    const int ii = rb * 8 + threadIdx.x;
    if (ii < n) {
      double M = -INFINITY, Sd = 0.0;
      for (int s2 = 0; s2 < P.nseg; ++s2) {
        const double2 q = __ldcg(&P.part64_row[(size_t)s2 * n + ii]);
        lse64_merge(M, Sd, q.x, q.y);
      }
      double* out = (mode == MODE_PLAIN) ? P.out_plain : (mode == MODE_EVAL ? nullptr : P.f[cf]);
      double* outA = (mode == MODE_PLAIN || mode == MODE_EVAL) ? nullptr : P.fA64[cf];
      double L;
      finish64(M, Sd, ii, P, P.f[cf], P.a, P.loga, out, outA, P.Lrow, accv, &st->numeric, &L);
      if (mode == MODE_PLAIN && P.logratio_plain) P.logratio_plain[ii] = L;
    }
  }
  block_sum3(accv, s_red);
  if (threadIdx.x == 0) {
    P.cnt_row[rb] = 0u;
    double* ab = P.acc_row + rb * 4;
    ab[0] = accv[0];
    ab[1] = accv[1];
    ab[2] = accv[2];
    __threadfence();
    const unsigned prev = atomicAdd(&P.gcnt[1], 1u);
    s_last = (prev == (unsigned)(P.nrowblk64 - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double tot[3];
  grid_sum3(P.acc_row, P.nrowblk64, tot, s_red);
  if (threadIdx.x == 0) {
    P.gcnt[1] = 0u;
    if (mode == MODE_EVAL) st->l1_row = tot[0];
    else final_step(P, mode == MODE_PLAIN ? MODE_PLAIN : MODE_SK_ROW, tot, cf);
  }
}

// eps-shifted float64 copies of a potential (level start, after f').
__global__ void shift64_kernel(const Prob* __restrict__ PP, const double* __restrict__ p,
                               const double* __restrict__ logw, int len, double* __restrict__ out) {
  const Prob& P = *PP;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x)
    out[i] = p[i] + P.eps * logw[i];
}

cudaError_t launch_col64(const Prob* dP, const Prob& hP, int mode, const AccArgs& a,
                         cudaStream_t s) {
  dim3 grid(hP.ncolblk64, mode == MODE_S4 ? 1 : hP.nstripe);
  col64_kernel<<<grid, 128, 0, s>>>(dP, mode, a);
  return cudaGetLastError();
}

cudaError_t launch_row64(const Prob* dP, const Prob& hP, int mode, cudaStream_t s) {
  dim3 grid(hP.nrowblk64, hP.nseg);
  row64_kernel<<<grid, 256, 0, s>>>(dP, mode);
  return cudaGetLastError();
}

cudaError_t launch_shift64(const Prob* dP, const double* p, const double* logw, int len,
                           double* out, cudaStream_t s) {
  const int blocks = (len + 255) / 256;
  shift64_kernel<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(dP, p, logw, len, out);
  return cudaGetLastError();
}

// The two exponentials of the float32 passes, elementwise, for accuracy
// checks: variant 0 is 2^(p + q) of the evaluation passes that verify a
// result (ex2_pq), variant 1 the hardware approximation of the iterations
// applied to the float32 sum p + q.
__global__ void exp2_check_kernel(int count, const float* __restrict__ p,
                                  const float* __restrict__ q, int variant,
                                  float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = variant == 0 ? ex2_pq(p[i], q[i]) : ex2_approx(__fadd_rn(p[i], q[i]));
}

cudaError_t launch_exp2_check(int count, const float* p, const float* q, int variant, float* out,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(((long long)count + 255) / 256, 4096);
  exp2_check_kernel<<<grid, 256, 0, s>>>(count, p, q, variant, out);
  return cudaGetLastError();
}

EOT_DEBUG_UNIT(passes)

}  // namespace eotk
