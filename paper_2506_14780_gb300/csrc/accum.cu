// Passes that accumulate a block of k vectors weighted by the coupling:
//
//  * Op(pi)^T Z (column direction, Eq. def_Op_pi_T):
//        out_j = sum_i exp((f_i + g_j - C_ij)/eps) a_i Z_i          (Z: n x k)
//  * Op(pi) Z (row direction, Eq. def_Op_pi):
//        out_i = sum_j exp((f_i + g_j - C_ij)/eps) b_j Z_j          (Z: m x k)
//  * the fused SK-NR column pass at f_k (Algorithm 4.1, value / gradient /
//    Hessian on V_l): with h = f_k^{C,eps} (the column transform, computed in
//    the same pass as a log-sum-exp),
//        W_j = sum_i pi(f_k, h)_ij V_i = b_j * softmax_i(x_ij) . V,
//    the semi-dual coupling of Eq. (dQ_semi) applied to the modes; plus the
//    marginal test of the iteration and the new column potential h.
//
// Exponents are formed exactly as in the Sinkhorn passes (eot_device.cuh).
// Column direction: one thread per column (warp = 32 consecutive columns, one
// 128-byte line per row), 8 warps interleaved over a stripe of rows, the stripe's
// rows of Z staged in shared memory and broadcast.  Row direction: a warp owns
// two rows, lanes stride along the columns, Z_j read per column and shared by
// the two rows.  Partial (reference, sum, k accumulators) per segment are
// combined in fixed order by the last-arriving CTA of each index block.
#include "eot_device.cuh"
#include "eot_internal.h"

namespace eotk {

enum AccMode : int { ACC_KCOL = 0, ACC_S4 = 1, ACC_KROW = 2 };



// ---------------------------------------------------------------------------
// Column direction (K-apply col, S4).
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(kThreads) colacc_kernel(AccArgs args) {
  const Prob& P = *args.P;
  State* st = P.st;
  const bool s4 = args.mode == ACC_S4;
  if (s4 && st->done) return;
  const int fb = s4 ? st->cur_f : args.fbuf;
  const int gb = s4 ? st->cur_g : args.gbuf;
  const int dst_g = (st->cur_g + 1) % 3;
  const float* __restrict__ rA = P.rs[fb].A;
  const float* __restrict__ rAL = P.rs[fb].AL;
  const float* __restrict__ cK = P.cs[gb].K;
  const float* __restrict__ cKL = P.cs[gb].KL;

  constexpr int CH = 64;          // rows per staged chunk
  constexpr int KS = K + 4;       // padded smem stride
  extern __shared__ float smem[];
  float* sZ = smem;                       // [CH][KS]
  float2* sRow = reinterpret_cast<float2*>(sZ + CH * KS);   // [CH]
  float* sRed = reinterpret_cast<float*>(sRow + CH);        // [8][32][K+2]
  __shared__ double s_red[24];
  __shared__ unsigned s_last;

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n = P.n, m = P.m, kk = args.k;
  const int cb = blockIdx.x, seg = blockIdx.y;
  const int j = cb * 32 + lane;
  const bool jv = j < m;
  const int i_beg = seg * args.seg_len;
  const int i_end = min(n, i_beg + args.seg_len);
  const float k2 = P.k2;
  const float Kj = jv ? cK[j] : P.M;
  const float cc0 = jv ? cKL[j] * k2 : 0.f;
  float cc = cc0;
  float ref = 0.f, run = -INFINITY, S = 0.f;
  float acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.f;

  for (int base = i_beg; base < i_end; base += CH) {
    const int nr = min(CH, i_end - base);
    __syncthreads();
    for (int t = threadIdx.x; t < CH * K; t += kThreads) {
      const int r = t / K, k = t - r * K;
      sZ[r * KS + k] = (r < nr && k < kk) ? args.Z[(size_t)(base + r) * kk + k] : 0.f;
    }
    if ((int)threadIdx.x < nr) sRow[threadIdx.x] = make_float2(rA[base + threadIdx.x], rAL[base + threadIdx.x]);
    __syncthreads();
    if (!jv) continue;
    for (int r = wid; r < nr; r += 8) {
      const float c = __ldg(P.C + (size_t)(base + r) * m + j);
      const float2 ra = sRow[r];
      const float t = __fadd_rn(split_exponent(c, Kj, ra.x), ra.y);
      float y = __fmaf_rn(t, k2, cc);
      if (y > run) {
        run = y;
        if (run > kRecenter || (run < -kRecenter && run > -INFINITY)) {
          const float d = rintf(run);
          S = scale2(S, -d);
#pragma unroll
          for (int k = 0; k < K; ++k) acc[k] = scale2(acc[k], -d);
          ref += d;
          cc = __fsub_rn(cc0, ref);
          run -= d;
          y = __fmaf_rn(t, k2, cc);
        }
      }
      const float e = ex2_approx(y);
      S += e;
      const float4* z4 = reinterpret_cast<const float4*>(sZ + r * KS);
#pragma unroll
      for (int k4 = 0; k4 < K / 4; ++k4) {
        const float4 z = z4[k4];
        acc[4 * k4 + 0] = __fmaf_rn(e, z.x, acc[4 * k4 + 0]);
        acc[4 * k4 + 1] = __fmaf_rn(e, z.y, acc[4 * k4 + 1]);
        acc[4 * k4 + 2] = __fmaf_rn(e, z.z, acc[4 * k4 + 2]);
        acc[4 * k4 + 3] = __fmaf_rn(e, z.w, acc[4 * k4 + 3]);
      }
    }
  }
  // intra-CTA combine over the 8 warps: rescale to the CTA maximum reference
  __syncthreads();
  {
    float* my = sRed + (wid * 32 + lane) * (K + 2);
    my[0] = (S > 0.f) ? ref : -INFINITY;
    my[1] = S;
#pragma unroll
    for (int k = 0; k < K; ++k) my[2 + k] = acc[k];
  }
  __syncthreads();
  // thread t: column t & 31, slice (t >> 5) of the K+2 entries
  {
    const int col = threadIdx.x & 31, sl = threadIdx.x >> 5;
    float R = -INFINITY;
    for (int w = 0; w < 8; ++w) R = fmaxf(R, sRed[(w * 32 + col) * (K + 2)]);
    const int jj = cb * 32 + col;
    for (int e = sl; e < K + 2; e += 8) {
      float v = 0.f;
      if (e == 0) {
        v = R;
      } else {
        for (int w = 0; w < 8; ++w) {
          const float* src = sRed + (w * 32 + col) * (K + 2);
          const float rw = src[0];
          if (rw == -INFINITY) continue;
          v += (rw == R) ? src[e] : scale2(src[e], rw - R);
        }
      }
      if (jj < m) args.part[((size_t)seg * m + jj) * (K + 2) + e] = v;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&args.cnt[cb], 1u);
    s_last = (prev == (unsigned)(args.nseg - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // --- combine the segments of the 32 columns of this block ---
  double accv[3] = {0.0, 0.0, 0.0};
  {
    const int col = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int jj = cb * 32 + col;
    if (jj < m) {
      float R = -INFINITY;
      for (int s = 0; s < args.nseg; ++s) {
        const float* src = args.part + ((size_t)s * m + jj) * (K + 2);
        if (__ldcg(src + 1) > 0.f) R = fmaxf(R, __ldcg(src));
      }
      double Stot = 0.0;
      for (int s = 0; s < args.nseg; ++s) {
        const float* src = args.part + ((size_t)s * m + jj) * (K + 2);
        const float Ss = __ldcg(src + 1);
        if (Ss > 0.f) {
          const float rs = __ldcg(src);
          Stot += (double)(rs == R ? Ss : scale2(Ss, rs - R));
        }
      }
      // out = scale * sum_s 2^(R_s - R) acc_s
      float scale;
      if (s4) scale = (float)(P.b[jj] / Stot);          // b_j * softmax normalisation
      else scale = scale2(1.f, R);                       // un-normalised K-apply
      for (int k = sl; k < kk; k += 8) {
        float v = 0.f;
        for (int s = 0; s < args.nseg; ++s) {
          const float* src = args.part + ((size_t)s * m + jj) * (K + 2);
          const float Ss = __ldcg(src + 1);
          if (Ss > 0.f) {
            const float rs = __ldcg(src);
            v += (rs == R) ? __ldcg(src + 2 + k) : scale2(__ldcg(src + 2 + k), rs - R);
          }
        }
        args.out[(size_t)jj * kk + k] = v * scale;
      }
      if (s4 && sl == 0) {
        // column transform h and the marginal test, as in the Sinkhorn column pass
        float L = R * kLn2 + log_sum(Stot);
        const double sh = P.g[gb][jj];
        double o = sh - P.eps * (double)L;
        if (!isfinite(o) || !(Stot > 0.0) || fabs(o) > P.pot_bound) {
          atomicAdd(&st->numeric, 1);
          o = sh;
          L = 0.f;
        }
        P.g[dst_g][jj] = o;
        P.Lcol[jj] = L;
        double hi;
        float lo;
        split_grid(o + P.eps * P.logb[jj], P.qscale, P.qinv, hi, lo);
        P.cs[dst_g].A[jj] = (float)(hi + (double)P.M);
        P.cs[dst_g].AL[jj] = lo;
        split_grid(o, P.qscale, P.qinv, hi, lo);
        P.cs[dst_g].K[jj] = (float)((double)P.M - hi);
        P.cs[dst_g].KL[jj] = lo;
        const double wj = P.b[jj];
        accv[0] = wj * (double)fabsf(expm1f(L));
        accv[1] = wj * (double)L;
        accv[2] = wj * o;
      }
    }
  }
  if (!s4) {
    if (threadIdx.x == 0) args.cnt[cb] = 0u;
    return;
  }
  // block sums (only warp 0 holds values) and the grid-final step
  {
    double v0 = warp_sum_d(accv[0]), v1 = warp_sum_d(accv[1]), v2 = warp_sum_d(accv[2]);
    if (threadIdx.x == 0) {
      args.cnt[cb] = 0u;
      double* ab = args.blkacc + cb * 4;
      ab[0] = v0;
      ab[1] = v1;
      ab[2] = v2;
      __threadfence();
      const unsigned prev = atomicAdd(args.gcnt, 1u);
      if (prev == (unsigned)(args.nblk - 1)) {
        __threadfence();
        *args.gcnt = 0u;
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int b2 = 0; b2 < args.nblk; ++b2) {
          t0 += __ldcg(&args.blkacc[b2 * 4 + 0]);
          t1 += __ldcg(&args.blkacc[b2 * 4 + 1]);
          t2 += __ldcg(&args.blkacc[b2 * 4 + 2]);
        }
        st->l1_col = t0;
        st->sum_wL = t1;
        st->qsemi = st->sum_af + t2;   // Q_semi(f_k) = <f_k, a> + <h, b>
        st->iter += 1;
        st->nr_ok = 0;
        if (st->numeric > 0) st->done = 3;
        else if (t0 < st->tol) st->done = 1;
        else if (st->iter >= st->max_iter) st->done = 2;
      }
    }
  }
  (void)s_red;
}

// ---------------------------------------------------------------------------
// Row direction (K-apply row): out_i = sum_j 2^{y_ij} Z_j, two rows per warp.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(kThreads) rowacc_kernel(AccArgs args) {
  const Prob& P = *args.P;
  const float* __restrict__ cA = P.cs[args.gbuf].A;
  const float* __restrict__ cAL = P.cs[args.gbuf].AL;
  const float* __restrict__ rK = P.rs[args.fbuf].K;
  const float* __restrict__ rKL = P.rs[args.fbuf].KL;
  constexpr int RW = (K <= 32) ? 2 : 1;
  extern __shared__ float smem[];
  float* sRed = smem;   // [8 warps][32 lanes][RW*(K+2)+1]
  constexpr int SR = RW * (K + 2) + 1;
  __shared__ unsigned s_last;

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n = P.n, m = P.m, kk = args.k;
  const int rb = blockIdx.x, seg = blockIdx.y;
  const int i0 = rb * (8 * RW) + wid * RW;
  const int c_beg = seg * args.seg_len;
  const int c_end = min(m, c_beg + args.seg_len);
  const float k2 = P.k2;
  float Kr[RW], cc0[RW], cc[RW], ref[RW], run[RW], S[RW];
  bool rv[RW];
  float acc[RW][K];
#pragma unroll
  for (int r = 0; r < RW; ++r) {
    const int i = i0 + r;
    rv[r] = i < n;
    Kr[r] = rv[r] ? rK[i] : P.M;
    cc0[r] = rv[r] ? rKL[i] * k2 : 0.f;
    cc[r] = cc0[r];
    ref[r] = 0.f;
    run[r] = -INFINITY;
    S[r] = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) acc[r][k] = 0.f;
  }
  if (rv[0]) {
    for (int j = c_beg + lane; j < c_end; j += 32) {
      const float ca = __ldg(cA + j), cal = __ldg(cAL + j);
      float e[RW];
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        if (!rv[r]) { e[r] = 0.f; continue; }
        const float c = __ldg(P.C + (size_t)(i0 + r) * m + j);
        const float t = __fadd_rn(split_exponent(c, Kr[r], ca), cal);
        float y = __fmaf_rn(t, k2, cc[r]);
        if (y > run[r]) {
          run[r] = y;
          if (run[r] > kRecenter || (run[r] < -kRecenter && run[r] > -INFINITY)) {
            const float d = rintf(run[r]);
            S[r] = scale2(S[r], -d);
#pragma unroll
            for (int k = 0; k < K; ++k) acc[r][k] = scale2(acc[r][k], -d);
            ref[r] += d;
            cc[r] = __fsub_rn(cc0[r], ref[r]);
            run[r] -= d;
            y = __fmaf_rn(t, k2, cc[r]);
          }
        }
        e[r] = ex2_approx(y);
        S[r] += e[r];
      }
      const float* zr = args.Z + (size_t)j * kk;
      if ((kk & 3) == 0) {
        const float4* z4 = reinterpret_cast<const float4*>(zr);
#pragma unroll
        for (int k4 = 0; k4 < K / 4; ++k4) {
          if (4 * k4 < kk) {
            const float4 z = __ldg(z4 + k4);
#pragma unroll
            for (int r = 0; r < RW; ++r) {
              acc[r][4 * k4 + 0] = __fmaf_rn(e[r], z.x, acc[r][4 * k4 + 0]);
              acc[r][4 * k4 + 1] = __fmaf_rn(e[r], z.y, acc[r][4 * k4 + 1]);
              acc[r][4 * k4 + 2] = __fmaf_rn(e[r], z.z, acc[r][4 * k4 + 2]);
              acc[r][4 * k4 + 3] = __fmaf_rn(e[r], z.w, acc[r][4 * k4 + 3]);
            }
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (k < kk) {
            const float z = __ldg(zr + k);
#pragma unroll
            for (int r = 0; r < RW; ++r) acc[r][k] = __fmaf_rn(e[r], z, acc[r][k]);
          }
        }
      }
    }
  }
  // warp reduction through shared memory: bring all lanes to the warp max ref
  float* my = sRed + (wid * 32 + lane) * SR;
#pragma unroll
  for (int r = 0; r < RW; ++r) {
    float R = (S[r] > 0.f) ? ref[r] : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) R = fmaxf(R, __shfl_xor_sync(0xffffffffu, R, o));
    const bool live = S[r] > 0.f;
    const float dr = (ref[r] == R) ? 0.f : ref[r] - R;
    my[r * (K + 2) + 0] = R;
    my[r * (K + 2) + 1] = live ? scale2(S[r], dr) : 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) my[r * (K + 2) + 2 + k] = live ? scale2(acc[r][k], dr) : 0.f;
  }
  __syncwarp();
  // lane l sums entries l, l+32, ... over the warp's 32 lanes
  for (int e = lane; e < RW * (K + 2); e += 32) {
    float v;
    if ((e % (K + 2)) == 0) {
      v = sRed[(wid * 32) * SR + e];
    } else {
      v = 0.f;
      for (int l = 0; l < 32; ++l) v += sRed[(wid * 32 + l) * SR + e];
    }
    const int r = e / (K + 2), q = e % (K + 2);
    const int i = i0 + r;
    if (i < n) args.part[((size_t)seg * n + i) * (K + 2) + q] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&args.cnt[rb], 1u);
    s_last = (prev == (unsigned)(args.nseg - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // combine the segments of the 8*RW rows of this block
  {
    constexpr int TPR = kThreads / (8 * RW);   // threads per row
    const int rr = threadIdx.x / TPR, sl = threadIdx.x % TPR;
    const int i = rb * (8 * RW) + rr;
    if (i < n) {
      float R = -INFINITY;
      for (int s = 0; s < args.nseg; ++s) {
        const float* src = args.part + ((size_t)s * n + i) * (K + 2);
        if (__ldcg(src + 1) > 0.f) R = fmaxf(R, __ldcg(src));
      }
      const float scale = scale2(1.f, R);
      for (int k = sl; k < kk; k += TPR) {
        float v = 0.f;
        for (int s = 0; s < args.nseg; ++s) {
          const float* src = args.part + ((size_t)s * n + i) * (K + 2);
          const float Ss = __ldcg(src + 1);
          if (Ss > 0.f) {
            const float rs = __ldcg(src);
            v += (rs == R) ? __ldcg(src + 2 + k) : scale2(__ldcg(src + 2 + k), rs - R);
          }
        }
        args.out[(size_t)i * kk + k] = v * scale;
      }
    }
  }
  if (threadIdx.x == 0) args.cnt[rb] = 0u;
}

// ---------------------------------------------------------------------------
template <int K>
static cudaError_t launch_colacc_k(const AccArgs& a, int ncolblk, cudaStream_t s) {
  constexpr int CH = 64, KS = K + 4;
  const size_t sm = (size_t)CH * KS * 4 + CH * 8 + (size_t)8 * 32 * (K + 2) * 4;
  dim3 grid(ncolblk, a.nseg);
  colacc_kernel<K><<<grid, kThreads, sm, s>>>(a);
  return cudaGetLastError();
}

template <int K>
static cudaError_t launch_rowacc_k(const AccArgs& a, int nrowblk, cudaStream_t s) {
  const size_t sm = (size_t)8 * 32 * ((K <= 32 ? 2 : 1) * (K + 2) + 1) * 4;
  dim3 grid(nrowblk, a.nseg);
  rowacc_kernel<K><<<grid, kThreads, sm, s>>>(a);
  return cudaGetLastError();
}

template <int K>
static void set_acc_attr() {
  constexpr int CH = 64, KS = K + 4;
  const size_t smc = (size_t)CH * KS * 4 + CH * 8 + (size_t)8 * 32 * (K + 2) * 4;
  cudaFuncSetAttribute(colacc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
  const size_t smr = (size_t)8 * 32 * ((K <= 32 ? 2 : 1) * (K + 2) + 1) * 4;
  cudaFuncSetAttribute(rowacc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
}

// Dynamic shared-memory limits of every instantiation (once per device, before
// any graph capture).
void init_acc_attributes() {
  set_acc_attr<16>();
  set_acc_attr<32>();
  set_acc_attr<48>();
  set_acc_attr<64>();
}

int acc_template_k(int k) { return k <= 16 ? 16 : k <= 32 ? 32 : k <= 48 ? 48 : 64; }

cudaError_t launch_colacc(const AccArgs& a, int ncolblk, cudaStream_t s) {
  switch (acc_template_k(a.k)) {
    case 16: return launch_colacc_k<16>(a, ncolblk, s);
    case 32: return launch_colacc_k<32>(a, ncolblk, s);
    case 48: return launch_colacc_k<48>(a, ncolblk, s);
    default: return launch_colacc_k<64>(a, ncolblk, s);
  }
}

cudaError_t launch_rowacc(const AccArgs& a, int nrowblk, cudaStream_t s) {
  switch (acc_template_k(a.k)) {
    case 16: return launch_rowacc_k<16>(a, nrowblk, s);
    case 32: return launch_rowacc_k<32>(a, nrowblk, s);
    case 48: return launch_rowacc_k<48>(a, nrowblk, s);
    default: return launch_rowacc_k<64>(a, nrowblk, s);
  }
}

}  // namespace eotk
