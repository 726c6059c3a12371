// Column-direction coupling products on the tensor cores (tcgen05, TMEM):
//
//   Op(pi)^T Z:  out_j = sum_i exp((f_i + g_j - C_ij)/eps) a_i Z_i  (Eq. def_Op_pi_T)
//   SK-NR fused column pass at f_k (Algorithm 4.1): h = f_k^{C,eps} by a
//   log-sum-exp and W_j = sum_i pi(f_k, h)_ij V_i, plus the marginal test, the
//   gradient weights d_j and per-block partials of W^T D_b^{-1} W, d^T W
//   (Eq. dQ_semi, d2Q_semi restricted to V).
//
// The contraction E^T Z with E_ij = 2^{y_ij} is a dense m x n x k product:
// a CTA owns 128 columns (the MMA's M) and a segment of rows, walked in chunks
// of 32 rows (4 MMAs of K = 8).  Its 256 threads form the exponentials exactly
// as the Sinkhorn passes do (two threads per column, 16 rows each), keep the
// column's running log-sum-exp, and write E as the A operand: each thread its
// own 64-byte piece of row "column j" of a K-major, 128-byte-swizzled tile.
// Z (V for SK-NR) enters as the B operand from pre-built swizzled tiles of the
// transposed rows.  Precision: every operand is split into TF32 hi + lo and the
// three products hi*hi + hi*lo + lo*hi are accumulated in float32 in TMEM
// (relative error ~1e-6, the accuracy of a float32 sum).  One thread issues the
// MMAs; two buffers let the tensor core work on chunk c while the threads form
// chunk c + 1; completion is tracked with tcgen05.commit on an mbarrier whose
// waits are bounded.
#include <algorithm>

#include "eot_device.cuh"
#include "eot_internal.h"
#include "reduce.cuh"
#include "tc.cuh"
#include "stream_common.cuh"

namespace eotk {

constexpr int kMmaM = 128;      // columns per CTA
constexpr int kMmaKC = 32;      // rows per chunk
constexpr int kMmaWait = 1 << 22;
constexpr int kMmaMaxCluster = 8;   // segments per output block merged in one cluster
constexpr double kNrRangeLn = 60.0 * 0.6931471805599453;   // |ln column sum| bound for the products

// Swizzled tiles of Z^T: for chunk c of 32 rows, tile (c, part) holds NN rows
// (the k index, padded with zeros) of 32 floats (the chunk's rows of Z), part 0
// the TF32-rounded value, part 1 the TF32-rounded remainder.
__global__ void build_tiles_kernel(const float* __restrict__ Z, int n, int kk, int NN,
                                   float* __restrict__ tiles, const int* __restrict__ skip) {
  pdl_enter();
  if (skip && *skip) return;
  if (!EOT_CHECK(kk >= 1 && kk <= NN, 201)) return;
  const int nch = (n + kMmaKC - 1) / kMmaKC;
  const long total = (long)nch * NN * kMmaKC;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int k = (int)(e % kMmaKC);
    const int r = (int)((e / kMmaKC) % NN);
    const int c = (int)(e / ((long)kMmaKC * NN));
    const int i = c * kMmaKC + k;
    const float v = (i < n && r < kk) ? Z[(size_t)i * kk + r] : 0.f;
    const float hi = to_tf32(v);
    const float lo = to_tf32(v - hi);
    const size_t off = sw128_off(r, k >> 2) / 4 + (k & 3);
    tiles[((size_t)c * 2 + 0) * NN * kMmaKC + off] = hi;
    tiles[((size_t)c * 2 + 1) * NN * kMmaKC + off] = lo;
  }
}

// Shared state of the segment-combining epilogue.
struct MmaEpi {
  double red[24];
  unsigned last;
};

// Epilogue of the CTA that arrived last on output block cb (128 columns, or
// 128 rows for the row-direction product; `len` = m or n): merge the
// segments' (reference, sum) heads and product rows of its 128 indices, write
// the product (or, in the SK-NR pass, W = pi(f_k, h)^T V with h = f_k^{C,eps},
// the new potential h and its split arrays, d_j, and the block partials of
// W^T D_b^{-1} W and d^T W; the last block takes the grid-wide step: L1
// test, Q_semi(f_k), iteration count).  Run by threads 0..255 (named barrier
// 1); `smem` is scratch of at least 2 * 128 (NN + 1) + 256 + 4608 floats.
template <int NN>
__device__ __noinline__ void colmma_finish(const AccArgs& args, const Prob& P, unsigned char* smem,
                              MmaEpi& epi, int cb, int gb, int dst_g, int len) {
  State* st = P.st;
  const bool s4 = args.mode == ACC_S4;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int m = len, kk = args.k;
  const int c = tid & (kMmaM - 1), h = tid >> 7;
  const int j = cb * kMmaM + c;
  const bool jv = j < m;
  constexpr int WS = NN + 1;                    // odd row stride
  float* sW = reinterpret_cast<float*>(smem);   // [128][NN + 1]  W_j
  float* sWb = sW + kMmaM * WS;                 // [128][NN + 1]  W_j / b_j
  float* sD = sWb + kMmaM * WS;                 // [128] d_j
  float* sS = sD + kMmaM;                       // [128] scale of the product row
  float* sP = sS + kMmaM;                       // [4][16 * 64] partial 4 x 4 blocks
  double accv[3] = {0.0, 0.0, 0.0};
  if (tid < kMmaM) {
    float R = -INFINITY;
    double Stot = 0.0;
    if (jv) merge_segments_k(args.part, args.nseg, m, NN + 4, j, R, Stot);
    // pi(f_k, h)^T V: the product rows times b_j / sum_i 2^{y_ij}
    sS[c] = (s4 && jv) ? (float)(P.b[j] / (Stot * ldexp(1.0, (int)R))) : 1.f;
    if (s4) {
      sD[c] = 0.f;
      if (jv) {
        double Ld = (double)R * 0.6931471805599453 + (double)log_sum(Stot);
        // The products hold the terms at their absolute scale 2^{y_ij}.  The
        // column's sum 2^R Stot lies between its largest term and n times it,
        // so a sum within 2^{+-60} keeps every term that matters inside the
        // float32 range; otherwise the Newton step is skipped.  (R itself is
        // the log-sum-exp reference, which may sit up to 64 below the largest
        // term, and says nothing about the range.)
        if (!(fabs(Ld) <= kNrRangeLn)) atomicOr(&st->nr_degenerate, 1);
        const double sh = P.g[gb][j];
        double o = sh - P.eps * Ld;
        if (!isfinite(o) || !(Stot > 0.0) || fabs(o) > P.pot_bound) {
          atomicAdd(&st->numeric, 1);
          o = sh;
          Ld = 0.0;
        }
        const float L = (float)Ld;
        P.g[dst_g][j] = o;
        P.Lcol[j] = L;
        double hi;
        float lo;
        split_grid(o + P.eps * P.logb[j], P.qscale, P.qinv, hi, lo);
        P.cs[dst_g].A[j] = (float)(hi + (double)P.M);
        P.cs[dst_g].AL[j] = lo;
        split_grid(o, P.qscale, P.qinv, hi, lo);
        P.cs[dst_g].K[j] = (float)((double)P.M - hi);
        P.cs[dst_g].KL[j] = lo;
        const double wj = P.b[j];
        const float em = expm1f(L);
        const double dj = -(double)em;          // 1 - exp((g_j - h_j)/eps)
        args.dw[j] = dj;
        sD[c] = (float)dj;
        accv[0] = wj * (double)fabsf(em);
        accv[1] = wj * Ld;
        accv[2] = wj * o;
      }
    }
  }
  cons_sync();
  // the product rows: thread (c, h) sums the segments of 16-value pieces
  // h, h + 2, ... of row c (segments in a fixed order)
  {
    const float scale = sS[c];
    const float binv = (s4 && jv) ? (float)(1.0 / P.b[j]) : 0.f;
#pragma unroll 1
    for (int k0 = 16 * h; k0 < NN; k0 += 32) {
      float acc[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) acc[k] = 0.f;
      if (jv) {
#pragma unroll 3
        for (int sg = 0; sg < args.nseg; ++sg) {
          const float4* src = reinterpret_cast<const float4*>(
              args.part + ((size_t)sg * m + j) * (NN + 4) + 4 + k0);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 v = __ldcg(src + q);
            acc[4 * q + 0] += v.x;
            acc[4 * q + 1] += v.y;
            acc[4 * q + 2] += v.z;
            acc[4 * q + 3] += v.w;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float wv = acc[k] * scale;
        if (k0 + k < kk && jv) args.out[(size_t)j * kk + k0 + k] = wv;
        if (s4) {
          const bool live = jv && k0 + k < kk;
          sW[c * WS + k0 + k] = live ? wv : 0.f;
          sWb[c * WS + k0 + k] = live ? wv * binv : 0.f;
        }
      }
    }
  }
  if (!s4) {
    if (tid == 0) args.cnt[cb] = 0u;
    return;
  }
  cons_sync();
  {
    // block partials of W^T D_b^{-1} W (4 x 4 register blocks; the 128
    // columns split among 256 / nb^2 thread groups) and d^T W, float32 sums
    // over the block's columns, float64 across blocks
    double* dstp = args.wtw_part + (size_t)cb * (kk * kk + kk);
    const int nb = (kk + 3) >> 2, nb2 = nb * nb;    // nb <= 12
    const int groups = nb2 <= 64 ? 4 : 2;           // each thread owns at most two blocks
    const int gsz = kStConsumers / groups;
    const int grp = tid / gsz, t = tid - grp * gsz;
    const int q0 = grp * (kMmaM / groups), q1 = q0 + kMmaM / groups;
    for (int blk = t; blk < nb2; blk += gsz) {
      const int br = blk / nb, bc = blk - br * nb;
      float o4[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) o4[x][y] = 0.f;
      for (int q = q0; q < q1; ++q) {
        float u[4], v[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          u[x] = sWb[q * WS + min(4 * br + x, NN - 1)];
          v[x] = sW[q * WS + min(4 * bc + x, NN - 1)];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) o4[x][y] = __fmaf_rn(u[x], v[y], o4[x][y]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) sP[(grp * nb2 + blk) * 16 + x * 4 + y] = o4[x][y];
    }
    // d^T W
    for (int r = tid; r < kk; r += kStConsumers) {
      float sdw = 0.f;
      for (int q = 0; q < kMmaM; ++q) sdw = __fmaf_rn(sD[q], sW[q * WS + r], sdw);
      dstp[kk * kk + r] = (double)sdw;
    }
    cons_sync();
    for (int e = tid; e < nb2 * 16; e += kStConsumers) {
      const int blk = e >> 4, x = (e >> 2) & 3, y = e & 3;
      const int br = blk / nb, bc = blk - br * nb;
      const int r = 4 * br + x, cc = 4 * bc + y;
      float sum = 0.f;
      for (int g2 = 0; g2 < groups; ++g2) sum += sP[(g2 * nb2 + blk) * 16 + x * 4 + y];
      if (r < kk && cc < kk) dstp[r * kk + cc] = (double)sum;
    }
  }
  // the block's three sums (only the first 128 threads hold nonzero values)
  cons_sum3(accv, epi.red, kMmaM);
  if (tid == 0) {
    args.cnt[cb] = 0u;
    double* ab = args.blkacc + cb * 4;
    ab[0] = accv[0];
    ab[1] = accv[1];
    ab[2] = accv[2];
    epi.last = arrive_count(args.gcnt) == (unsigned)(args.nblk - 1);
  }
  cons_sync();
  if (!epi.last || wid != 0) return;
  double tot[3];
  warp0_grid_sum3(args.blkacc, args.nblk, tot);
  if (lane == 0) {
    *args.gcnt = 0u;
    st->l1_col = tot[0];
    st->sum_wL = tot[1];
    st->qsemi = st->sum_af + tot[2];   // Q_semi(f_k) = <f_k, a> + <h, b>
    st->iter += 1;
    trace_test(P, st, st->iter, tot[0], st->qsemi);
    st->nr_ok = 0;
    if (st->numeric > 0) st->done = 3;
    else st->done = stop_code(st, tot[0], st->iter, st->tol, st->max_iter, P.stall_window);
  }
}

// ---------------------------------------------------------------------------
// Cluster epilogue of the staged kernel: the nseg segment CTAs of an output
// block form one thread-block cluster.  Each CTA leaves its record (per
// output index: the (reference, sum) head of its log-sum-exp and its product
// row) in its own shared memory; after a cluster barrier, CTA rank r merges
// the records of all segments for its slice of the block's 128 indices by
// distributed shared-memory loads (segments in rank order: deterministic),
// finishes those indices (the product or W = pi(f_k, h)^T V, and in the SK-NR
// pass h = f_k^{C,eps}, its splits, d_j) and, in the SK-NR pass, the slice's
// partials of W^T D_b^{-1} W, d^T W and the three scalar sums; after a second
// barrier rank 0 adds the slices' partials (rank order) into the block's
// record and takes the grid-wide step as the last block to arrive.  No
// global round trip between the segments' streams and the merge.
// Shared memory (from the 1024-aligned base; the cost and operand rings are
// idle by then): records [128][NN + 4] floats (R, -, S as a double, the
// product row), then the slice rows and the partials.
// ---------------------------------------------------------------------------
template <int NN>
struct ClusterEpi {
  static constexpr int RW = NN + 4;                               // record floats
  static constexpr int WS = NN + 1;                               // slice row stride
  static constexpr uint32_t rec = 128u * RW * 4u;
  static constexpr uint32_t scr = rec;                            // sW, sWb [128][WS]
  static constexpr uint32_t vec = scr + 2u * 128u * WS * 4u;      // sD, sS, sBi [128]
  static constexpr uint32_t part = (vec + 3u * 128u * 4u + 15u) & ~15u;   // doubles
  static constexpr uint32_t bytes_s4 = part + (uint32_t)(NN * NN + NN + 4) * 8u;
  static constexpr uint32_t bytes_prod = scr + 3u * 128u * 4u + 128u * NN * 4u;
};

template <int NN>
__device__ __noinline__ void cluster_finish(const AccArgs& args, const Prob& P,
                                            unsigned char* sbase, uint32_t sb, MmaEpi& epi,
                                            int cb, int gb, int dst_g, int len, bool s4) {
  using CE = ClusterEpi<NN>;
  State* st = P.st;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int kk = args.k;
  const int cs = (int)gridDim.y;
  const int rank = (int)cluster_rank();
  const int c0 = rank * kMmaM / cs, c1 = (rank + 1) * kMmaM / cs, w = c1 - c0;
  float* sW = reinterpret_cast<float*>(sbase + CE::scr);
  float* sWb = sW + kMmaM * CE::WS;
  float* sD = reinterpret_cast<float*>(sbase + (s4 ? CE::vec : CE::scr));
  float* sS = sD + kMmaM;
  float* sBi = sS + kMmaM;
  double accv[3] = {0.0, 0.0, 0.0};
  // heads: one thread per index of the slice, every segment's head in flight
  if (tid < w) {
    const int cc = c0 + tid, j = cb * kMmaM + cc;
    const bool jv = j < len;
    float rr[8];
    double ss[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if (r < cs) {
        const uint32_t a = peer_addr(sb + (uint32_t)(cc * CE::RW) * 4u, (uint32_t)r);
        rr[r] = ld_peer_f(a);
        ss[r] = ld_peer_d(a + 8u);
      }
    }
    float R = -INFINITY;
    double Stot = 0.0;
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (r < cs) merge_dd(R, Stot, rr[r], ss[r]);
    sS[tid] = (s4 && jv) ? (float)(P.b[j] / (Stot * ldexp(1.0, (int)R))) : 1.f;
    sBi[tid] = (s4 && jv) ? (float)(1.0 / P.b[j]) : 0.f;
    if (s4) {
      sD[tid] = 0.f;
      if (jv) {
        double Ld = (double)R * 0.6931471805599453 + (double)log_sum(Stot);
        // The products hold the terms at their absolute scale 2^{y_ij}.  The
        // column's sum 2^R Stot lies between its largest term and n times it,
        // so a sum within 2^{+-60} keeps every term that matters inside the
        // float32 range; otherwise the Newton step is skipped.  (R itself is
        // the log-sum-exp reference, which may sit up to 64 below the largest
        // term, and says nothing about the range.)
        if (!(fabs(Ld) <= kNrRangeLn)) atomicOr(&st->nr_degenerate, 1);
        const double sh = P.g[gb][j];
        double o = sh - P.eps * Ld;
        if (!isfinite(o) || !(Stot > 0.0) || fabs(o) > P.pot_bound) {
          atomicAdd(&st->numeric, 1);
          o = sh;
          Ld = 0.0;
        }
        const float L = (float)Ld;
        P.g[dst_g][j] = o;
        P.Lcol[j] = L;
        double hi;
        float lo;
        split_grid(o + P.eps * P.logb[j], P.qscale, P.qinv, hi, lo);
        P.cs[dst_g].A[j] = (float)(hi + (double)P.M);
        P.cs[dst_g].AL[j] = lo;
        split_grid(o, P.qscale, P.qinv, hi, lo);
        P.cs[dst_g].K[j] = (float)((double)P.M - hi);
        P.cs[dst_g].KL[j] = lo;
        const double wj = P.b[j];
        const float em = expm1f(L);
        const double dj = -(double)em;          // 1 - exp((g_j - h_j)/eps)
        args.dw[j] = dj;
        sD[tid] = (float)dj;
        accv[0] = wj * (double)fabsf(em);
        accv[1] = wj * Ld;
        accv[2] = wj * o;
      }
    }
  }
  // product rows of the slice: float4 pieces, segments in rank order
  {
    constexpr int Q4 = NN / 4;
    float* raw = s4 ? sW : reinterpret_cast<float*>(sbase + CE::scr + 3u * 128u * 4u);
    for (int e = tid; e < w * Q4; e += nthr) {
      const int t = e / Q4, q = e - t * Q4;
      const uint32_t off = sb + (uint32_t)((c0 + t) * CE::RW + 4 + 4 * q) * 4u;
      float4 v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < cs) v[r] = ld_peer4(peer_addr(off, (uint32_t)r));
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        if (r < cs) {
          acc.x += v[r].x;
          acc.y += v[r].y;
          acc.z += v[r].z;
          acc.w += v[r].w;
        }
      }
      if (s4) {
        float* dstw = sW + t * CE::WS + 4 * q;
        dstw[0] = acc.x;
        dstw[1] = acc.y;
        dstw[2] = acc.z;
        dstw[3] = acc.w;
      } else {
        reinterpret_cast<float4*>(raw)[t * Q4 + q] = acc;
      }
    }
  }
  __syncthreads();
  // scale the rows: W_j (SK-NR: times b_j / sum_i 2^{y_ij}; products: absolute)
  {
    const float* raw = s4 ? sW : reinterpret_cast<const float*>(sbase + CE::scr + 3u * 128u * 4u);
    for (int e = tid; e < w * NN; e += nthr) {
      const int t = e / NN, k = e - t * NN;
      const int j = cb * kMmaM + c0 + t;
      const bool live = j < len && k < kk;
      const float wv = (s4 ? raw[t * CE::WS + k] : raw[t * NN + k]) * sS[t];
      if (live) args.out[(size_t)j * kk + k] = wv;
      if (s4) {
        sW[t * CE::WS + k] = live ? wv : 0.f;
        sWb[t * CE::WS + k] = live ? wv * sBi[t] : 0.f;
      }
    }
  }
  if (!s4) {
    // every peer has read this CTA's records before any CTA leaves
    cluster_sync_all();
    return;
  }
  __syncthreads();
  // the slice's partials: W^T D_b^{-1} W and d^T W (float32 over the slice's
  // indices, in index order) and the three scalar sums (float64)
  double* part = reinterpret_cast<double*>(sbase + CE::part);
  const int cnt = kk * kk + kk;
  for (int e = tid; e < kk * kk; e += nthr) {
    const int r = e / kk, c2 = e - r * kk;
    float sum = 0.f;
    for (int t = 0; t < w; ++t) sum = __fmaf_rn(sWb[t * CE::WS + r], sW[t * CE::WS + c2], sum);
    part[e] = (double)sum;
  }
  for (int e = tid; e < kk; e += nthr) {
    float sum = 0.f;
    for (int t = 0; t < w; ++t) sum = __fmaf_rn(sD[t], sW[t * CE::WS + e], sum);
    part[kk * kk + e] = (double)sum;
  }
  if (wid < 4) {   // the slice's indices live in threads 0..w-1 (w <= 128)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double x = warp_sum_d(accv[k]);
      if (lane == 0) epi.red[k * 8 + wid] = x;
    }
  }
  __syncthreads();
  if (tid < 3) part[cnt + tid] = (epi.red[tid * 8] + epi.red[tid * 8 + 1]) +
                                 (epi.red[tid * 8 + 2] + epi.red[tid * 8 + 3]);
  // every slice's partials are in place, and every record has been read
  cluster_sync_all();
  if (rank == 0) {
    const uint32_t pa = sb + CE::part;
    double* dstp = args.wtw_part + (size_t)cb * cnt;
    for (int e = tid; e < cnt + 3; e += nthr) {
      double v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < cs) v[r] = ld_peer_d(peer_addr(pa + (uint32_t)e * 8u, (uint32_t)r));
      double sum = 0.0;
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < cs) sum += v[r];
      if (e < cnt) dstp[e] = sum;
      else args.blkacc[cb * 4 + (e - cnt)] = sum;
    }
    __syncthreads();
    if (tid == 0) epi.last = arrive_count(args.gcnt) == (unsigned)(args.nblk - 1);
    __syncthreads();
    if (epi.last && wid == 0) {
      double tot[3];
      warp0_grid_sum3(args.blkacc, args.nblk, tot);
      if (lane == 0) {
        *args.gcnt = 0u;
        st->l1_col = tot[0];
        st->sum_wL = tot[1];
        st->qsemi = st->sum_af + tot[2];   // Q_semi(f_k) = <f_k, a> + <h, b>
        st->iter += 1;
        trace_test(P, st, st->iter, tot[0], st->qsemi);
        st->nr_ok = 0;
        if (st->numeric > 0) st->done = 3;
        else st->done = stop_code(st, tot[0], st->iter, st->tol, st->max_iter, P.stall_window);
      }
    }
  }
  // rank 0 has read every slice's partials before any CTA leaves
  cluster_sync_all();
}

template <int NN>
struct MmaSmem {
  static constexpr size_t a_tile = (size_t)kMmaM * 128;           // 16 KB
  static constexpr size_t b_tile = (size_t)NN * 128;
  static constexpr size_t a_off = 0;                              // [2 buf][hi, lo]
  static constexpr size_t b_off = 4 * a_tile;                     // [2 buf][hi, lo]
  static constexpr size_t row_off = b_off + 4 * b_tile;           // [2][32] float2
  static constexpr size_t bytes = row_off + 2 * 32 * 8 + 1024;    // + alignment slack
};

template <int NN>
__global__ void __launch_bounds__(256) colmma_kernel(AccArgs args, const float* __restrict__ tiles) {
  pdl_enter();
  const Prob& P = *args.P;
  State* st = P.st;
  const bool s4 = args.mode == ACC_S4;
  if (s4 && st->done) return;
  if (args.skip && *args.skip) return;
  if (!EOT_CHECK(args.k >= 1 && args.k <= NN, 202)) return;
  const int fb = s4 ? st->cur_f : args.fbuf;
  const int gb = s4 ? st->cur_g : args.gbuf;
  const int dst_g = (st->cur_g + 1) % 3;
  const float* __restrict__ rA = P.rs[fb].A;
  const float* __restrict__ rAL = P.rs[fb].AL;
  const float* __restrict__ cK = P.cs[gb].K;
  const float* __restrict__ cKL = P.cs[gb].KL;
  using SM = MmaSmem<NN>;

  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t s_mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ float s_lr[2][kMmaM];
  __shared__ double s_ls[2][kMmaM];
  __shared__ MmaEpi epi;
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sbase = smem_raw + (base - raw);
  float2* sRow = reinterpret_cast<float2*>(sbase + SM::row_off);

  const int tid = threadIdx.x, wid = tid >> 5;
  const int c = tid & (kMmaM - 1), h = tid >> 7;     // column within the tile, row half
  const int n = P.n, m = P.m;
  const int cb = blockIdx.x, seg = blockIdx.y;
  const int j = cb * kMmaM + c;
  const bool jv = j < m;
  const int i_beg = seg * args.seg_len;
  const int i_end = min(n, i_beg + args.seg_len);
  const int nch = (i_end - i_beg + kMmaKC - 1) / kMmaKC;
  const int gch0 = i_beg / kMmaKC;                   // global chunk index of chunk 0
  const float k2 = P.k2;
  const float Kj = jv ? cK[j] : P.M;
  const float cc0 = jv ? cKL[j] * k2 : 0.f;
  float ref = 0.f, run = -INFINITY, S = 0.f, Sc = 0.f;   // run: maximum of y - ref
  constexpr uint32_t idesc = idesc_tf32(kMmaM, NN);
  constexpr uint32_t tcols = NN <= 32 ? 32 : (NN <= 64 ? 64 : 128);
  constexpr int BV = (2 * NN * kMmaKC) / (4 * 256);  // float4 of B tiles per thread per chunk

  if (tid == 0) {
    mbar_init(smem_addr(&s_mbar[0]), 1);
    mbar_init(smem_addr(&s_mbar[1]), 1);
    mbar_init_fence();
    s_err = 0;
  }
  if (wid == 0) tmem_alloc(smem_addr(&s_tmem), tcols);

  // ---- prefetch registers ----
  float cn[16];
  float2 rn = make_float2(0.f, 0.f);
  float4 bn[BV > 0 ? BV : 1];
  auto fetch = [&](int ch) {
    const int base_i = i_beg + ch * kMmaKC;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int i = base_i + h * 16 + u;
      cn[u] = (jv && i < i_end) ? __ldg(P.C + (size_t)i * m + j) : 0.f;
    }
    if (tid < kMmaKC) {
      const int i = base_i + tid;
      rn = i < i_end ? make_float2(__ldg(rA + i), __ldg(rAL + i)) : make_float2(0.f, 0.f);
    }
    const float4* src = reinterpret_cast<const float4*>(tiles + (size_t)(gch0 + ch) * 2 * NN * kMmaKC);
#pragma unroll
    for (int q = 0; q < BV; ++q) bn[q] = __ldg(src + tid + q * 256);
  };
  auto publish = [&](int buf) {
    float4* dstb = reinterpret_cast<float4*>(sbase + SM::b_off + (size_t)buf * 2 * SM::b_tile);
#pragma unroll
    for (int q = 0; q < BV; ++q) dstb[tid + q * 256] = bn[q];
    if (tid < kMmaKC) sRow[buf * kMmaKC + tid] = rn;
  };
  if (nch > 0) {
    fetch(0);
    publish(0);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t mbar0 = smem_addr(&s_mbar[0]), mbar1 = smem_addr(&s_mbar[1]);

  int last_issued = -1;
  for (int ch = 0; ch < nch; ++ch) {
    const int buf = ch & 1;
    last_issued = ch;
    float cv[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) cv[u] = cn[u];
    if (ch + 1 < nch) fetch(ch + 1);
    const int base_i = i_beg + ch * kMmaKC;
    // exponentials of this thread's 16 rows, written as A (hi and lo tiles)
    float ew[16];
    float part = 0.f;   // the current group of 4 terms, added to S compensated
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int r = h * 16 + u;
      ew[u] = 0.f;
      if (jv && base_i + r < i_end) {
        const float2 ra = sRow[buf * kMmaKC + r];
        const float t = __fadd_rn(split_exponent(cv[u], Kj, ra.x), ra.y);
        const float y = __fmaf_rn(t, k2, cc0);   // relative to the column's shift
        float z = ref == 0.f ? y : __fsub_rn(y, ref);
        if (z > run) {
          run = z;
          if (needs_move(run, ref)) {
            // the Sinkhorn passes' reference rule (exact power-of-two
            // rescaling; the reference returns to 0 once the maximum is
            // within the window), so that the dominant terms carry no
            // rounding of a large exponent
            S = __fadd_rn(__fsub_rn(S, Sc), part);
            Sc = 0.f;
            part = 0.f;
            move_ref(run, ref, S);
            z = ref == 0.f ? y : __fsub_rn(y, ref);
          }
        }
        const float e = ex2_approx(z);
        part += e;
        ew[u] = (ref == 0.f) ? e : scale2(e, ref);   // absolute scale for the product
      }
      if ((u & 3) == 3) {
        // Kahan: a serial float32 sum over a long segment would floor the
        // L1 marginal test
        const float yk = __fsub_rn(part, Sc);
        const float tk = __fadd_rn(S, yk);
        Sc = __fsub_rn(__fsub_rn(tk, S), yk);
        S = tk;
        part = 0.f;
      }
    }
    {
      unsigned char* ahi = sbase + SM::a_off + (size_t)buf * 2 * SM::a_tile;
      unsigned char* alo = ahi + SM::a_tile;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float4 vh, vl;
        vh.x = to_tf32(ew[4 * q + 0]); vl.x = to_tf32(ew[4 * q + 0] - vh.x);
        vh.y = to_tf32(ew[4 * q + 1]); vl.y = to_tf32(ew[4 * q + 1] - vh.y);
        vh.z = to_tf32(ew[4 * q + 2]); vl.z = to_tf32(ew[4 * q + 2] - vh.z);
        vh.w = to_tf32(ew[4 * q + 3]); vl.w = to_tf32(ew[4 * q + 3] - vh.w);
        const uint32_t off = sw128_off(c, h * 4 + q);
        *reinterpret_cast<float4*>(ahi + off) = vh;
        *reinterpret_cast<float4*>(alo + off) = vl;
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ahi = base + (uint32_t)(SM::a_off + (size_t)buf * 2 * SM::a_tile);
      const uint32_t alo = ahi + (uint32_t)SM::a_tile;
      const uint32_t bhi = base + (uint32_t)(SM::b_off + (size_t)buf * 2 * SM::b_tile);
      const uint32_t blo = bhi + (uint32_t)SM::b_tile;
#pragma unroll
      for (int s = 0; s < kMmaKC / 8; ++s) {
        const uint32_t ko = s * 32;
        mma_tf32(tmem, sdesc_sw128(ahi + ko), sdesc_sw128(bhi + ko), idesc, (ch > 0 || s > 0) ? 1u : 0u);
        mma_tf32(tmem, sdesc_sw128(ahi + ko), sdesc_sw128(blo + ko), idesc, 1u);
        mma_tf32(tmem, sdesc_sw128(alo + ko), sdesc_sw128(bhi + ko), idesc, 1u);
      }
      mma_commit(buf ? mbar1 : mbar0);
    }
    if (ch + 1 < nch) {
      const int nb = buf ^ 1;
      if (ch >= 1) {   // chunk ch - 1 used buffer nb: wait for its products
        if (!mbar_wait(nb ? mbar1 : mbar0, ((ch - 1) >> 1) & 1, kMmaWait)) s_err = 1;
      }
      publish(nb);
      fence_async_smem();
      __syncthreads();
      if (s_err) break;
    }
  }
  // all products done (or, after a failed wait, given a bounded chance to
  // finish) before the accumulator is read and TMEM is released
  bool ok = true;
  if (last_issued >= 0) {
    const int l1 = last_issued;
    ok = mbar_wait((l1 & 1) ? mbar1 : mbar0, (l1 >> 1) & 1, kMmaWait);
    if (l1 >= 1) {
      const int l2 = l1 - 1;
      ok = mbar_wait((l2 & 1) ? mbar1 : mbar0, (l2 >> 1) & 1, kMmaWait) && ok;
    }
  }
  if (!ok) s_err = 1;
  tc_fence_after();
  S = __fsub_rn(S, Sc);
  // LSE halves -> one state per column
  s_lr[h][c] = (S > 0.f) ? ref : -INFINITY;
  s_ls[h][c] = (double)S;
  __syncthreads();
  const bool err = s_err != 0;
  if (tid < kMmaM) {
    float R = -INFINITY;
    double Sd = 0.0;
    merge_d(R, Sd, s_lr[0][c], (float)s_ls[0][c]);
    merge_d(R, Sd, s_lr[1][c], (float)s_ls[1][c]);
    float* dst = args.part + ((size_t)seg * m + (jv ? j : 0)) * (NN + 4);
    // accumulator row c lives in TMEM lane c (warp w reads lanes 32w..32w+31)
#pragma unroll
    for (int q = 0; q < NN / 16; ++q) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(wid * 32) << 16) + q * 16, v);
      if (jv) {
#pragma unroll
        for (int u = 0; u < 16; ++u) dst[4 + q * 16 + u] = (err || nch == 0) ? 0.f : v[u];
      }
    }
    if (jv) {
      dst[0] = R;
      dst[1] = (float)Sd;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 0) tmem_dealloc(tmem, tcols);
  if (err && tid == 0) atomicAdd(&st->numeric, 1);
  if (tid == 0) epi.last = arrive_count(&args.cnt[cb]) == (unsigned)(args.nseg - 1);
  __syncthreads();
  if (!epi.last) return;
  colmma_finish<NN>(args, P, sbase, epi, cb, gb, dst_g, m);
}

// ---------------------------------------------------------------------------
// Staged variant for costs with 16-byte aligned rows (a 2-D tensor map of C):
// warp-specialised, A operand in TMEM.
//   * warp 8 (producer): per chunk of 32 rows, one tiled tensor copy of the
//     32 x 128 cost tile, one bulk copy of the chunk's B tiles (hi, lo) and
//     two of the rows' split coefficients into a ring of stages;
//   * warps 0..7 (consumers): thread (c, h) forms the 16 exponents of column
//     c, rows 16h..16h+15 of the chunk, from shared memory (two rows at a
//     time with the packed float32x2 instructions), keeps the column's running
//     log-sum-exp, and stores the exponentials' TF32 hi / lo parts with
//     tcgen05.st into TMEM lane c (columns = the chunk's rows): the A operand
//     of the next MMAs, no shared-memory round trip;
//   * warp 9 (MMA issuer, TMEM owner): 4 x 3 MMAs per chunk (K = 8; hi*hi,
//     hi*lo, lo*hi) from the TMEM A buffer and the B tiles in shared memory.
// Three TMEM A buffers let the consumers run up to two chunks ahead of the
// tensor core.  Barriers: full[s] / empty[s] of the cost ring (copies landed;
// 8 consumer warps read them), bfull[t] / bempty[t] of the operand ring
// (copy landed; MMA commit), afull[b] (8 consumer warps stored A), aempty[b]
// (MMA commit), acc (all MMAs done).  The producer warp feeds the cost ring,
// the MMA thread the operand ring.  Every wait is bounded.
// ---------------------------------------------------------------------------
constexpr int kTmThreads = 320;
constexpr uint32_t kTmTile = kMmaKC * kMmaM * 4;   // 16 KB cost tile
constexpr uint32_t kTmA = 64;                      // TMEM column of A buffer 0
constexpr int kTmNA = 3;                           // TMEM A buffers (64 columns each)
constexpr uint32_t kTmCols = 256;

// Two rings: cost stages (tile + the rows' coefficients), released by the
// consumers as soon as they have read them, and operand stages (B hi, B lo),
// released by the MMA commit.
template <int NN>
struct TmaSmem {
  static constexpr int cstages = 4;
  static constexpr int bstages = NN <= 48 ? 3 : 2;
  static constexpr uint32_t coef_off = kTmTile;                     // A[32], AL[32]
  static constexpr uint32_t cstage = (kTmTile + 256 + 1023) / 1024 * 1024;
  static constexpr uint32_t bstage = 2 * NN * 128;                  // a multiple of 1024
  static constexpr uint32_t b_base = cstages * cstage;
  static constexpr size_t bytes = (size_t)b_base + (size_t)bstages * bstage + 1024;
  static constexpr uint32_t ctx = kTmTile + 256;
};

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t v[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// D (TMEM) += A (TMEM, M x 8 tf32 at column ta) * B (shared memory descriptor)^T
__device__ __forceinline__ void mma_tf32_ts(uint32_t tmem_d, uint32_t ta, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
      "r"(ta), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// TF32 parts of a pair of non-negative floats: hi = x with the 13 low fraction
// bits cleared, lo = x - hi (exact in float32).  The tensor core reads a tf32
// operand from the high 19 bits of its 32-bit register, so lo is passed whole
// and enters with its leading 11 bits: hi + lo as multiplied matches x to
// 2^-21 relative.
__device__ __forceinline__ void tf32_split2(float2 x, uint32_t& h0, uint32_t& h1, uint32_t& l0,
                                            uint32_t& l1) {
  h0 = __float_as_uint(x.x) & 0xFFFFE000u;
  h1 = __float_as_uint(x.y) & 0xFFFFE000u;
  const float2 lo = __ffma2_rn(f2(__uint_as_float(h0), __uint_as_float(h1)), f2(-1.f, -1.f), x);
  l0 = __float_as_uint(lo.x);
  l1 = __float_as_uint(lo.y);
}

// ROW = false: column direction (output index j over 128-column blocks,
// reduction over rows i; the cost tile is 32 rows x 128 columns).  ROW = true:
// the row-direction product Op(pi) Z, out_i = sum_j 2^{y_ij} Z_j at absolute
// scale (Eq. def_Op_pi); output index i over 128-row blocks, reduction over
// columns j, the cost tile 128 rows x 32 columns from a second tensor map with
// 128-byte swizzle (16-byte chunk q of row r at chunk q ^ (r & 7)), so that a
// thread reads its row's 16 values with four conflict-free 16-byte loads.
template <int NN, bool ROW, bool CL>
__global__ void __launch_bounds__(kTmThreads, 2)
    mma_tma_kernel(AccArgs args, const float* __restrict__ tiles) {
  static_assert(ClusterEpi<NN>::bytes_prod + 1024 <= TmaSmem<NN>::bytes, "epilogue smem");
  static_assert(NN > 48 || ClusterEpi<NN>::bytes_s4 + 1024 <= TmaSmem<NN>::bytes, "epilogue smem");
  pdl_enter();
  const Prob* PP = args.P;
  const Prob& P = *PP;
  State* st = P.st;
  const bool s4 = !ROW && args.mode == ACC_S4;
  if (s4 && st->done) return;
  if (!EOT_CHECK(args.k >= 1 && args.k <= NN, 203)) return;
  if (args.skip && *args.skip) return;   // uniform over the grid (and any cluster)
  const int fb = s4 ? st->cur_f : args.fbuf;
  const int gb = s4 ? st->cur_g : args.gbuf;
  const int dst_g = (st->cur_g + 1) % 3;
  using SM = TmaSmem<NN>;
  constexpr int NS = SM::cstages, NB = SM::bstages;

  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[NS];
  __shared__ __align__(8) uint64_t empty_bar[NS];
  __shared__ __align__(8) uint64_t bfull[NB];
  __shared__ __align__(8) uint64_t bempty[NB];
  __shared__ __align__(8) uint64_t afull[kTmNA];
  __shared__ __align__(8) uint64_t aempty[kTmNA];
  __shared__ __align__(8) uint64_t accf;
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ float s_lr[2][kMmaM];
  __shared__ double s_ls[2][kMmaM];
  __shared__ MmaEpi epi;
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sbase = smem_raw + (base - raw);

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = P.n, m = P.m;
  const int olen = ROW ? n : m;     // output indices
  const int rlen = ROW ? m : n;     // reduction indices
  const int cb = blockIdx.x, seg = blockIdx.y;
  const int i_beg = seg * args.seg_len;   // reduction range of this segment
  const int i_end = min(rlen, i_beg + args.seg_len);
  const int nch = i_end > i_beg ? (i_end - i_beg + kMmaKC - 1) / kMmaKC : 0;
  constexpr uint32_t idesc = idesc_tf32(kMmaM, NN);

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_addr(&full_bar[s]), 1);
      mbar_init(smem_addr(&empty_bar[s]), 8);
    }
    for (int t = 0; t < NB; ++t) {
      mbar_init(smem_addr(&bfull[t]), 1);
      mbar_init(smem_addr(&bempty[t]), 1);
    }
    for (int b = 0; b < kTmNA; ++b) {
      mbar_init(smem_addr(&afull[b]), 8);
      mbar_init(smem_addr(&aempty[b]), 1);
    }
    mbar_init(smem_addr(&accf), 1);
    mbar_init_fence();
    s_err = 0;
  }
  if (wid == 9) tmem_alloc(smem_addr(&s_tmem), kTmCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (wid == 8) {
    // ---------------- producer ----------------
    if (lane == 0) {
      // cost ring
      const float* rA = ROW ? P.cs[gb].A : P.rs[fb].A;
      const float* rAL = ROW ? P.cs[gb].AL : P.rs[fb].AL;
      int issued = 0;
      for (int ch = 0; ch < nch; ++ch) {
        const int s = ch % NS;
        if (ch >= NS &&
            !mbar_wait(smem_addr(&empty_bar[s]), ((ch / NS) - 1) & 1, kMmaWait)) {
          s_err = 1;
          break;
        }
        const uint32_t fbar = smem_addr(&full_bar[s]);
        const uint32_t dst = base + (uint32_t)s * SM::cstage;
        const int i0 = i_beg + ch * kMmaKC;   // a multiple of 32 (segments are)
        mbar_expect_tx(fbar, SM::ctx);
        // the box's first column (cb * 128, or i0) starts on a 16-byte boundary
        if (ROW)
          tma_load_2d(dst, &PP->tmCr, i0, cb * kMmaM, fbar);
        else
          tma_load_2d(dst, &PP->tmC, cb * kMmaM, i0, fbar);
        // the split arrays are padded to a multiple of 128 floats
        bulk_load(dst + SM::coef_off, rA + i0, 128u, fbar);
        bulk_load(dst + SM::coef_off + 128u, rAL + i0, 128u, fbar);
        ++issued;
      }
      // every copy has landed before the CTA may exit
      for (int s = 0; s < NS && s < issued; ++s) {
        const int last = s + ((issued - 1 - s) / NS) * NS;
        if (!mbar_wait(smem_addr(&full_bar[s]), (last / NS) & 1, kMmaWait)) s_err = 1;
      }
    }
  } else if (wid == 9) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      // operand ring: the MMA thread refills a stage once its own products
      // that read it are done (the consumers run well behind the tensor core)
      auto load_b = [&](int ch) {
        const int t = ch % NB;
        const uint32_t bbar = smem_addr(&bfull[t]);
        mbar_expect_tx(bbar, SM::bstage);
        bulk_load(base + SM::b_base + (uint32_t)t * SM::bstage,
                  tiles + (size_t)((i_beg + ch * kMmaKC) / kMmaKC) * 2 * NN * kMmaKC, SM::bstage,
                  bbar);
      };
      int bissued = 0;
      for (; bissued < NB && bissued < nch; ++bissued) load_b(bissued);
      for (int ch = 0; ch < nch; ++ch) {
        const int t = ch % NB, b = ch % kTmNA;
        if (!mbar_wait(smem_addr(&bfull[t]), (ch / NB) & 1, kMmaWait) ||
            !mbar_wait(smem_addr(&afull[b]), (ch / kTmNA) & 1, kMmaWait)) {
          s_err = 1;
          break;
        }
        tc_fence_after();
        const uint32_t bhi = base + SM::b_base + (uint32_t)t * SM::bstage;
        const uint32_t blo = bhi + (uint32_t)NN * 128u;
        const uint32_t ahi = tmem + kTmA + 64u * b, alo = ahi + 32u;
#pragma unroll
        for (int k = 0; k < kMmaKC / 8; ++k) {
          const uint32_t ko = k * 32;   // bytes of 8 tf32 in a B row
          mma_tf32_ts(tmem, ahi + 8 * k, sdesc_sw128(bhi + ko), idesc, (ch > 0 || k > 0) ? 1u : 0u);
          mma_tf32_ts(tmem, ahi + 8 * k, sdesc_sw128(blo + ko), idesc, 1u);
          mma_tf32_ts(tmem, alo + 8 * k, sdesc_sw128(bhi + ko), idesc, 1u);
        }
        mma_commit(smem_addr(&bempty[t]));
        mma_commit(smem_addr(&aempty[b]));
        if (bissued < nch) {
          if (!mbar_wait(smem_addr(&bempty[t]), (ch / NB) & 1, kMmaWait)) {
            s_err = 1;
            break;
          }
          load_b(bissued++);
        }
      }
      mma_commit(smem_addr(&accf));   // tracks every MMA issued above
      // every operand copy has landed before the CTA may exit
      for (int t = 0; t < NB && t < bissued; ++t) {
        const int last = t + ((bissued - 1 - t) / NB) * NB;
        if (!mbar_wait(smem_addr(&bfull[t]), (last / NB) & 1, kMmaWait)) s_err = 1;
      }
    }
  } else {
    // ---------------- consumers ----------------
    const int c = tid & (kMmaM - 1), h = tid >> 7;
    const int j = cb * kMmaM + c;       // output index (column, or row for ROW)
    const bool jv = j < olen;
    const float k2 = P.k2;
    const float2 k2v = f2(k2, k2), m1 = f2(-1.f, -1.f);
    const Split& os = ROW ? P.rs[fb] : P.cs[gb];
    const float Kj = jv ? os.K[j] : P.M;
    const float ccj = jv ? os.KL[j] * k2 : 0.f;
    const float2 nK2 = f2(-Kj, -Kj), cc2 = f2(ccj, ccj);
    const uint32_t tlane = (uint32_t)((wid & 3) * 32) << 16;
    float ref = 0.f, rr = -INFINITY, pscale = 1.f;
    float2 S2 = f2(0.f, 0.f), C2 = f2(0.f, 0.f);   // running sum, compensation
    bool werr = false;
    for (int ch = 0; ch < nch; ++ch) {
      const int s = ch % NS, b = ch % kTmNA;
      if (!__all_sync(0xffffffffu, mbar_wait(smem_addr(&full_bar[s]), (ch / NS) & 1, kMmaWait))) {
        werr = true;
        break;
      }
      const unsigned char* stg = sbase + (size_t)s * SM::cstage;
      const float* tile = reinterpret_cast<const float*>(stg);
      const float4* cA = reinterpret_cast<const float4*>(stg + SM::coef_off) + h * 4;
      const float4* cAL = reinterpret_cast<const float4*>(stg + SM::coef_off + 128) + h * 4;
      float2 y[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 av = cA[q], alv = cAL[q];
        float2 c0, c1;
        if (ROW) {
          const float4 cv = reinterpret_cast<const float4*>(tile)[c * 8 + ((h * 4 + q) ^ (c & 7))];
          c0 = f2(cv.x, cv.y);
          c1 = f2(cv.z, cv.w);
        } else {
          const int r = h * 16 + 4 * q;
          c0 = f2(tile[(r + 0) * kMmaM + c], tile[(r + 1) * kMmaM + c]);
          c1 = f2(tile[(r + 2) * kMmaM + c], tile[(r + 3) * kMmaM + c]);
        }
        const float2 t0 = __ffma2_rn(c0, m1, __fadd2_rn(f2(av.x, av.y), nK2));
        const float2 t1 = __ffma2_rn(c1, m1, __fadd2_rn(f2(av.z, av.w), nK2));
        y[2 * q + 0] = __ffma2_rn(t0, k2v, __ffma2_rn(f2(alv.x, alv.y), k2v, cc2));
        y[2 * q + 1] = __ffma2_rn(t1, k2v, __ffma2_rn(f2(alv.z, alv.w), k2v, cc2));
      }
      const int r0 = i_beg + ch * kMmaKC + h * 16;
      if (!jv || r0 + 16 > i_end) {
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          y[p].x = (jv && r0 + 2 * p < i_end) ? y[p].x : -INFINITY;
          y[p].y = (jv && r0 + 2 * p + 1 < i_end) ? y[p].y : -INFINITY;
        }
      }
      // the stage's cost and coefficients are read
      __syncwarp();
      if (lane == 0) mbar_arrive1(smem_addr(&empty_bar[s]));
      float2 z[8];
      const float2 nr = f2(-ref, -ref);
#pragma unroll
      for (int p = 0; p < 8; ++p) z[p] = ref == 0.f ? y[p] : __fadd2_rn(y[p], nr);
      float mx = fmaxf(fmaxf(fmaxf(z[0].x, z[0].y), fmaxf(z[1].x, z[1].y)),
                       fmaxf(fmaxf(z[2].x, z[2].y), fmaxf(z[3].x, z[3].y)));
      mx = fmaxf(mx, fmaxf(fmaxf(fmaxf(z[4].x, z[4].y), fmaxf(z[5].x, z[5].y)),
                           fmaxf(fmaxf(z[6].x, z[6].y), fmaxf(z[7].x, z[7].y))));
      rr = fmaxf(rr, mx);
      if (rr > -INFINITY && needs_move(rr, ref)) {
        kahan_fold2(S2, C2);
        float Ss = S2.x + S2.y;
        move_ref(rr, ref, Ss);
        S2 = f2(Ss, 0.f);
        pscale = scale2(1.f, ref);
        const float2 nr2 = f2(-ref, -ref);
#pragma unroll
        for (int p = 0; p < 8; ++p) z[p] = __fadd2_rn(y[p], nr2);
      }
      float2 e[8];
#pragma unroll
      for (int p = 0; p < 8; ++p) e[p] = ex2_2(z[p]);
      kahan_add2(S2, C2, __fadd2_rn(__fadd2_rn(__fadd2_rn(e[0], e[1]), __fadd2_rn(e[2], e[3])),
                                    __fadd2_rn(__fadd2_rn(e[4], e[5]), __fadd2_rn(e[6], e[7]))));
      if (ref != 0.f) {   // the product needs the terms at their absolute scale
        const float2 ps = f2(pscale, pscale);
#pragma unroll
        for (int p = 0; p < 8; ++p) e[p] = __fmul2_rn(e[p], ps);
      }
      uint32_t hv[16], lv[16];
#pragma unroll
      for (int p = 0; p < 8; ++p) tf32_split2(e[p], hv[2 * p], hv[2 * p + 1], lv[2 * p], lv[2 * p + 1]);
      // A buffer b is free once the MMAs of chunk ch - kTmNA are done
      if (ch >= kTmNA &&
          !__all_sync(0xffffffffu,
                      mbar_wait(smem_addr(&aempty[b]), ((ch - kTmNA) / kTmNA) & 1, kMmaWait))) {
        werr = true;
        break;
      }
      tc_fence_after();
      const uint32_t ta = tmem + tlane + kTmA + 64u * b + 16u * h;
      tmem_st16(ta, hv);
      tmem_st16(ta + 32u, lv);
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive1(smem_addr(&afull[b]));
    }
    // all products done (bounded) before the accumulator is read
    if (!__all_sync(0xffffffffu, mbar_wait(smem_addr(&accf), 0, kMmaWait))) werr = true;
    if (werr && lane == 0) s_err = 1;
    tc_fence_after();
    const double S = ((double)S2.x - (double)C2.x) + ((double)S2.y - (double)C2.y);
    s_lr[h][c] = (S > 0.0) ? ref : -INFINITY;
    s_ls[h][c] = S;
    cons_sync();
    if (tid < kMmaM) {
      float R = -INFINITY;
      double Sd = 0.0;
      merge_dd(R, Sd, s_lr[0][c], s_ls[0][c]);
      merge_dd(R, Sd, s_lr[1][c], s_ls[1][c]);
      if (CL) {
        // the record stays in this CTA's shared memory (the rings are idle:
        // every copy has landed and been consumed, every product is done)
        float* rec = reinterpret_cast<float*>(sbase) + c * (NN + 4);
#pragma unroll
        for (int q = 0; q < NN / 16; ++q) {
          float v[16];
          tmem_ld16(tmem + tlane + q * 16, v);
#pragma unroll
          for (int u = 0; u < 16; ++u) rec[4 + q * 16 + u] = (!jv || nch == 0) ? 0.f : v[u];
        }
        rec[0] = jv ? R : -INFINITY;
        *reinterpret_cast<double*>(rec + 2) = jv ? Sd : 0.0;
      }
      float* dst = args.part + ((size_t)seg * olen + (jv ? j : 0)) * (NN + 4);
      // accumulator row c lives in TMEM lane c (warp w reads lanes 32w..32w+31)
      if (!CL) {
#pragma unroll
        for (int q = 0; q < NN / 16; ++q) {
          float v[16];
          tmem_ld16(tmem + tlane + q * 16, v);
          if (jv) {
#pragma unroll
            for (int u = 0; u < 16; ++u) dst[4 + q * 16 + u] = nch == 0 ? 0.f : v[u];
          }
        }
        if (jv) {
          dst[0] = R;
          dst[1] = (float)Sd;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 9) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmCols);
  }
  if (CL) {
    // every warp of every CTA of the cluster takes the barriers below
    if (tid == 0 && s_err) atomicAdd(&st->numeric, 1);
    cluster_sync_all();   // every segment's record is in place
    cluster_finish<NN>(args, P, sbase, base, epi, cb, gb, dst_g, olen, s4);
    return;
  }
  if (wid >= 8) return;
  if (tid == 0) {
    if (s_err) atomicAdd(&st->numeric, 1);
    epi.last = arrive_count(&args.cnt[cb]) == (unsigned)(args.nseg - 1);
  }
  cons_sync();
  if (!epi.last) return;
  colmma_finish<NN>(args, P, sbase, epi, cb, gb, dst_g, olen);
}

// ---------------------------------------------------------------------------
int mma_width(int k) { return k <= 16 ? 16 : k <= 32 ? 32 : k <= 48 ? 48 : 64; }

int mma_record(int k) { return mma_width(k) + 4; }

size_t mma_tiles_floats(int n, int k) {
  return (size_t)((n + kMmaKC - 1) / kMmaKC) * 2 * mma_width(k) * kMmaKC;
}

// Segments merged through a thread-block cluster when the plan asks for it
// and an output block has at most 8 of them (the portable cluster size);
// otherwise through global records and the block's last-arriving CTA.
static bool mma_cluster_merge(const AccArgs& a, int nseg) {
  return a.cluster && nseg >= 1 && nseg <= kMmaMaxCluster;
}

// (A programmatic dependent launch of this kernel measured slower: its CTAs
// then hold shared memory and TMEM while the preceding pass finishes.)
template <int NN, bool ROW>
static cudaError_t launch_tma(const AccArgs& a, const float* tiles, dim3 grid, cudaStream_t s) {
  if (!mma_cluster_merge(a, (int)grid.y))
    return launch_pdl(mma_tma_kernel<NN, ROW, false>, grid, dim3(kTmThreads), TmaSmem<NN>::bytes,
                      s, a, tiles);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kTmThreads);
  cfg.dynamicSmemBytes = TmaSmem<NN>::bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = grid.y;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, mma_tma_kernel<NN, ROW, true>, a, tiles);
}

template <int NN>
static cudaError_t launch_colmma_k(const AccArgs& a, bool tma, const float* tiles, int ncolblk,
                                   cudaStream_t s) {
  dim3 grid(ncolblk, a.nseg);
  if (tma) return launch_tma<NN, false>(a, tiles, grid, s);
  return launch_pdl(colmma_kernel<NN>, grid, dim3(256), MmaSmem<NN>::bytes, s, a, tiles);
}

// The staged kernel needs the cost's tensor map (rows 16-byte aligned) and
// segments of whole 32-row chunks.
cudaError_t launch_colmma(const AccArgs& a, const Prob& hP, const float* tiles, int ncolblk,
                          cudaStream_t s) {
  const bool tma = hP.has_tmC && a.seg_len % kMmaKC == 0;
  switch (mma_width(a.k)) {
    case 16: return launch_colmma_k<16>(a, tma, tiles, ncolblk, s);
    case 32: return launch_colmma_k<32>(a, tma, tiles, ncolblk, s);
    case 48: return launch_colmma_k<48>(a, tma, tiles, ncolblk, s);
    default: return launch_colmma_k<64>(a, tma, tiles, ncolblk, s);
  }
}

// Row-direction product on the tensor cores (needs the cost's tensor maps;
// segments of whole 32-column chunks, output blocks of 128 rows).
cudaError_t launch_rowmma(const AccArgs& a, const float* tiles, int nrowblk, cudaStream_t s) {
  dim3 grid(nrowblk, a.nseg);
  if (a.seg_len % kMmaKC != 0) return cudaErrorInvalidValue;
  switch (mma_width(a.k)) {
    case 16: return launch_tma<16, true>(a, tiles, grid, s);
    case 32: return launch_tma<32, true>(a, tiles, grid, s);
    case 48: return launch_tma<48, true>(a, tiles, grid, s);
    default: return launch_tma<64, true>(a, tiles, grid, s);
  }
}

cudaError_t launch_build_tiles(const float* Z, int n, int kk, float* tiles, cudaStream_t s,
                               const int* skip) {
  const int NN = mma_width(kk);
  const long total = (long)((n + kMmaKC - 1) / kMmaKC) * NN * kMmaKC;
  const int blocks = (int)((total + 255) / 256);
  return launch_pdl(build_tiles_kernel, dim3(blocks < 4096 ? blocks : 4096), dim3(256), 0, s, Z, n,
                    kk, NN, tiles, skip);
}

template <int NN>
static void set_tma_attr() {
  // two CTAs per SM need most of the SM's shared memory
  cudaFuncSetAttribute(mma_tma_kernel<NN, false, false>,
                       cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  cudaFuncSetAttribute(mma_tma_kernel<NN, true, false>,
                       cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  cudaFuncSetAttribute(mma_tma_kernel<NN, false, true>,
                       cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  cudaFuncSetAttribute(mma_tma_kernel<NN, true, true>,
                       cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  cudaFuncSetAttribute(mma_tma_kernel<NN, false, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TmaSmem<NN>::bytes);
  cudaFuncSetAttribute(mma_tma_kernel<NN, true, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TmaSmem<NN>::bytes);
  cudaFuncSetAttribute(mma_tma_kernel<NN, false, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TmaSmem<NN>::bytes);
  cudaFuncSetAttribute(mma_tma_kernel<NN, true, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TmaSmem<NN>::bytes);
}

void init_mma_attributes() {
  cudaFuncSetAttribute(colmma_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)MmaSmem<16>::bytes);
  cudaFuncSetAttribute(colmma_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)MmaSmem<32>::bytes);
  cudaFuncSetAttribute(colmma_kernel<48>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)MmaSmem<48>::bytes);
  cudaFuncSetAttribute(colmma_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)MmaSmem<64>::bytes);
  set_tma_attr<16>();
  set_tma_attr<32>();
  set_tma_attr<48>();
  set_tma_attr<64>();
}

EOT_DEBUG_UNIT(mma)

}  // namespace eotk
