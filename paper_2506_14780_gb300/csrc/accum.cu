// Row-direction product on the CUDA cores, for costs without a tensor map (a
// row pitch that is not a multiple of 16 bytes):
//
//  * Op(pi) Z (Eq. def_Op_pi):
//        out_i = sum_j exp((f_i + g_j - C_ij)/eps) b_j Z_j          (Z: m x k)
//
// Exponents are formed exactly as in the Sinkhorn passes (eot_device.cuh).  A
// warp owns one or two rows, lanes stride along the columns, chunks of 128
// columns of Z are staged in shared memory (double buffered, conflict-free
// padding) and shared by the CTA's warps.  Partial (reference, sum, k
// accumulators) per segment are merged in parallel and in fixed order by the
// last-arriving CTA of each row block.  Also here: the reduction of the SK-NR
// column pass's per-block partials of W^T D_b^{-1} W and d^T W (Eq. d2Q_semi,
// dQ_semi on V), whose column pass itself runs on the tensor cores (mma.cu).
#include "eot_device.cuh"
#include "eot_internal.h"
#include "reduce.cuh"

namespace eotk {

constexpr int kCC = 128;  // columns per chunk (row direction)

template <int K>
struct RowAccSmem {
  static constexpr int RW = (K <= 32) ? 2 : 1;
  static constexpr int KS = K + 4;
  static constexpr size_t tiles = (size_t)2 * (kCC * KS + 2 * kCC) * 4;
  static constexpr size_t red = (size_t)8 * 32 * (RW * (K + 2) + 1) * 4;
  static constexpr size_t bytes = tiles > red ? tiles : red;
};

// Sum of the per-block partials of W^T D_b^{-1} W and sum_j d_j W_j: a CTA owns
// 32 entries, its 8 warps take interleaved blocks, the warps' sums are added in
// a fixed order.
__global__ void __launch_bounds__(256) wtw_reduce_kernel(const AccArgs args,
                                                         double* __restrict__ WtW,
                                                         double* __restrict__ gw) {
  pdl_enter();
  const State* st = args.P->st;
  if (st->done) return;
  __shared__ double sh[8][32];
  const int kk = args.k, cnt = kk * kk + kk;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (e < cnt) {
    for (int b0 = wid; b0 < args.nblk; b0 += 32) {
      double v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int b = b0 + 8 * q;
        v[q] = b < args.nblk ? __ldcg(&args.wtw_part[(size_t)b * cnt + e]) : 0.0;
      }
      s += (v[0] + v[1]) + (v[2] + v[3]);
    }
  }
  sh[wid][lane] = s;
  __syncthreads();
  if (wid == 0 && e < cnt) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += sh[w][lane];
    if (e < kk * kk) WtW[e] = t;
    else gw[e - kk * kk] = t;
  }
}

// ---------------------------------------------------------------------------
// Row direction (K-apply row): out_i = sum_j 2^{y_ij} Z_j.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(kThreads) rowacc_kernel(AccArgs args) {
  pdl_enter();
  if (args.skip && *args.skip) return;
  if (!EOT_CHECK(args.k >= 1 && args.k <= K, 501)) return;
  const Prob& P = *args.P;
  const float* __restrict__ cA = P.cs[args.gbuf].A;
  const float* __restrict__ cAL = P.cs[args.gbuf].AL;
  const float* __restrict__ rK = P.rs[args.fbuf].K;
  const float* __restrict__ rKL = P.rs[args.fbuf].KL;
  using SM = RowAccSmem<K>;
  constexpr int RW = SM::RW;
  constexpr int KS = SM::KS;
  constexpr int VPT = (kCC * K) / kThreads;   // staged Z values per thread per chunk
  extern __shared__ __align__(16) float smem[];
  float* sZ = smem;                                            // [2][kCC][KS]
  float2* sCol = reinterpret_cast<float2*>(smem + 2 * kCC * KS);  // [2][kCC]
  float* sRed = smem;                                          // reused after the loop
  constexpr int SR = RW * (K + 2) + 1;
  __shared__ unsigned s_last;

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n = P.n, m = P.m, kk = args.k;
  const int rb = blockIdx.x, seg = blockIdx.y;
  const int i0 = rb * (8 * RW) + wid * RW;
  const int c_beg = seg * args.seg_len;
  const int c_end = min(m, c_beg + args.seg_len);
  const int nchunks = (c_end - c_beg + kCC - 1) / kCC;
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
  float zn[VPT];
  float2 coln = make_float2(0.f, 0.f);
  float cn[RW][4];
  auto fetch = [&](int ch) {
    const int base = c_beg + ch * kCC;
    const int nc = min(kCC, c_end - base);
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
      const int t = threadIdx.x + q * kThreads;
      const int c = t / K, k = t - c * K;
      zn[q] = (c < nc && k < kk) ? __ldg(args.Z + (size_t)(base + c) * kk + k) : 0.f;
    }
    if ((int)threadIdx.x < nc)
      coln = make_float2(__ldg(cA + base + threadIdx.x), __ldg(cAL + base + threadIdx.x));
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = lane + 32 * q;
        cn[r][q] = (rv[r] && c < nc) ? __ldg(P.C + (size_t)(i0 + r) * m + base + c) : 0.f;
      }
  };
  auto publish = [&](int buf) {
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
      const int t = threadIdx.x + q * kThreads;
      const int c = t / K, k = t - c * K;
      sZ[(buf * kCC + c) * KS + k] = zn[q];
    }
    if ((int)threadIdx.x < kCC) sCol[buf * kCC + threadIdx.x] = coln;
  };
  if (nchunks > 0) {
    fetch(0);
    publish(0);
  }
  __syncthreads();
  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    const int nc = min(kCC, c_end - (c_beg + ch * kCC));
    float cv[RW][4];
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) cv[r][q] = cn[r][q];
    if (ch + 1 < nchunks) fetch(ch + 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lane + 32 * q;
      if (c < nc) {
        const float2 ca = sCol[buf * kCC + c];
        float e[RW];
#pragma unroll
        for (int r = 0; r < RW; ++r) {
          if (!rv[r]) {
            e[r] = 0.f;
            continue;
          }
          const float t = __fadd_rn(split_exponent(cv[r][q], Kr[r], ca.x), ca.y);
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
        const float4* z4 = reinterpret_cast<const float4*>(sZ + (buf * kCC + c) * KS);
#pragma unroll
        for (int k4 = 0; k4 < K / 4; ++k4) {
          const float4 z = z4[k4];
#pragma unroll
          for (int r = 0; r < RW; ++r) {
            acc[r][4 * k4 + 0] = __fmaf_rn(e[r], z.x, acc[r][4 * k4 + 0]);
            acc[r][4 * k4 + 1] = __fmaf_rn(e[r], z.y, acc[r][4 * k4 + 1]);
            acc[r][4 * k4 + 2] = __fmaf_rn(e[r], z.z, acc[r][4 * k4 + 2]);
            acc[r][4 * k4 + 3] = __fmaf_rn(e[r], z.w, acc[r][4 * k4 + 3]);
          }
        }
      }
    }
    if (ch + 1 < nchunks) publish(buf ^ 1);
    __syncthreads();
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
      double Stot = 0.0;
      merge_segments_k(args.part, args.nseg, n, K + 2, i, R, Stot);
      const float scale = scale2(1.f, R);
      for (int k = sl; k < kk; k += TPR) {
        float v = 0.f;
        for (int s0 = 0; s0 < args.nseg; s0 += 4) {
          float pr[4], pv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int s = s0 + q;
            const float* src = args.part + ((size_t)s * n + i) * (K + 2);
            pr[q] = s < args.nseg ? __ldcg(src) : -INFINITY;
            pv[q] = s < args.nseg ? __ldcg(src + 2 + k) : 0.f;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (pr[q] > -INFINITY) v += (pr[q] == R) ? pv[q] : scale2(pv[q], pr[q] - R);
        }
        args.out[(size_t)i * kk + k] = v * scale;
      }
    }
  }
  if (threadIdx.x == 0) args.cnt[rb] = 0u;
}

// ---------------------------------------------------------------------------
template <int K>
static cudaError_t launch_rowacc_k(const AccArgs& a, int nrowblk, cudaStream_t s) {
  dim3 grid(nrowblk, a.nseg);
  launch_pdl(rowacc_kernel<K>, dim3(grid), dim3(kThreads), RowAccSmem<K>::bytes, s, a);
  return cudaGetLastError();
}

template <int K>
static void set_acc_attr() {
  cudaFuncSetAttribute(rowacc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)RowAccSmem<K>::bytes);
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

// Rows per CTA of the row-direction product for a given width.
int rowacc_rows(int k) { return acc_template_k(k) <= 32 ? 16 : 8; }

cudaError_t launch_rowacc(const AccArgs& a, int nrowblk, cudaStream_t s) {
  switch (acc_template_k(a.k)) {
    case 16: return launch_rowacc_k<16>(a, nrowblk, s);
    case 32: return launch_rowacc_k<32>(a, nrowblk, s);
    case 48: return launch_rowacc_k<48>(a, nrowblk, s);
    default: return launch_rowacc_k<64>(a, nrowblk, s);
  }
}

cudaError_t launch_wtw_reduce(const AccArgs& a, double* WtW, double* gw, cudaStream_t s) {
  const int cnt = a.k * a.k + a.k;
  launch_pdl(wtw_reduce_kernel, dim3((cnt + 31) / 32), dim3(256), 0, s, a, WtW, gw);
  return cudaGetLastError();
}

EOT_DEBUG_UNIT(accum)

}  // namespace eotk
