// Small dense algebra on the device for SK-NR(l) (Algorithm 4.1) and the mode
// computation (Sec. 4), plus the O(n l) vector updates.
//
//  * weighted Gram partials/reduction:  G = A^T diag(w) B (+ w^T A), float32
//    products summed in float32 over 64-row chunks, float64 across chunks;
//  * newton_kernel (one CTA, float64): H_V = -(1/eps) [V^T D_a V - W^T D_b^{-1} W]
//    (Eq. d2Q_semi restricted to V_l with D_r ~ D_a, or exact with D_r),
//    grad_V = -sum_j d_j W_j with d_j = 1 - exp((g_j - h_j)/eps) (the semi-dual
//    gradient a - pi(f_k, h) 1 of Eq. dQ_semi projected on V; the row marginals
//    of pi(f_k, g_k) are exactly a after the row half-step), Cholesky of -H_V,
//    Delta = (-H_V)^{-1} grad_V; a failed factorisation rejects the step;
//  * fprime_kernel: f' = f_k + V Delta and its split arrays;
//  * eig_small_kernel (one CTA, float32 Jacobi): Rayleigh-Ritz of the block
//    subspace iteration and the Cholesky-QR transform of the next block;
//  * apply_kernel: Z <- (X - 1 c^T) B.
#include "eot_device.cuh"
#include "eot_internal.h"

namespace eotk {

constexpr int kGChunk = 64;

// part[chunk][p*p] (+ vpart[chunk][p] = sum_i vw_i A_i) partial sums over the
// rows of one chunk.
__global__ void __launch_bounds__(256) wgram_partial_kernel(
    const float* __restrict__ A, const float* __restrict__ B, const double* __restrict__ w,
    int wmode /*0: w, 1: 1/w*/, int len, int p, const double* __restrict__ vw,
    const float* __restrict__ vsrc, double* __restrict__ part, double* __restrict__ vpart,
    const State* st, int respect_done) {
  if (respect_done && st->done) return;
  extern __shared__ float sm[];
  float* sA = sm;                       // [kGChunk][p]
  float* sB = sA + kGChunk * p;         // [kGChunk][p]
  float* sw = sB + kGChunk * p;         // [kGChunk]
  float* svw = sw + kGChunk;            // [kGChunk]
  const int chunk = blockIdx.x;
  const int r0 = chunk * kGChunk;
  const int nr = min(kGChunk, len - r0);
  for (int t = threadIdx.x; t < kGChunk * p; t += blockDim.x) {
    const int r = t / p;
    sA[t] = r < nr ? A[(size_t)r0 * p + t] : 0.f;
    sB[t] = r < nr ? B[(size_t)r0 * p + t] : 0.f;
  }
  for (int r = threadIdx.x; r < kGChunk; r += blockDim.x) {
    float wv = 0.f, vv = 0.f;
    if (r < nr) {
      const double x = w[r0 + r];
      wv = (float)(wmode ? 1.0 / x : x);
      vv = vw ? (float)vw[r0 + r] : 0.f;
    }
    sw[r] = wv;
    svw[r] = vv;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int k = e / p, l = e - k * p;
    float s = 0.f;
    for (int r = 0; r < nr; ++r) s = __fmaf_rn(sw[r] * sA[r * p + k], sB[r * p + l], s);
    part[(size_t)chunk * p * p + e] = (double)s;
  }
  if (vpart) {
    for (int k = threadIdx.x; k < p; k += blockDim.x) {
      float s = 0.f;
      for (int r = 0; r < nr; ++r) s = __fmaf_rn(svw[r], sA[r * p + k], s);
      vpart[(size_t)chunk * p + k] = (double)s;
    }
  }
}

__global__ void wgram_reduce_kernel(const double* __restrict__ part, int nchunk, int cnt,
                                    double* __restrict__ out, const State* st, int respect_done) {
  if (respect_done && st->done) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= cnt) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * cnt + e];
  out[e] = s;
}

// ---------------------------------------------------------------------------
// Newton step on V (one warp, float64).  GV = V^T D_a V (or V^T D_r V),
// WtW = sum_j W_j W_j^T / b_j, gw = sum_j d_j W_j (d_j = -expm1(L_j)),
// Va = V^T a.  -H_V = (GV - WtW)/eps is factorised by a right-looking Cholesky
// with lanes over rows; Delta = (-H_V)^{-1} grad_V, grad_V = -gw.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) newton_kernel(const Prob* __restrict__ PP,
                                                    const double* __restrict__ WtW,
                                                    const double* __restrict__ gw,
                                                    const double* __restrict__ Dr) {
  const Prob& P = *PP;
  State* st = P.st;
  if (st->done) return;
  const int l = P.ell;
  const int lane = threadIdx.x;
  // the matrix is assembled in float64 (the difference GV - WtW cancels), the
  // factorisation and solves run in float32 (relative error ~1e-7 x cond)
  __shared__ float H[kMaxK * kMaxK];
  __shared__ float g[kMaxK];
  const double inv_eps = 1.0 / P.eps;
  for (int e = lane; e < l * l; e += 32) {
    const int r = e / l, c = e - r * l;
    const double gv = Dr ? 0.5 * (Dr[r * l + c] + Dr[c * l + r]) : 0.5 * (P.GV[r * l + c] + P.GV[c * l + r]);
    const double wt = 0.5 * (WtW[r * l + c] + WtW[c * l + r]);
    H[e] = (float)(inv_eps * (gv - wt));
  }
  for (int k = lane; k < l; k += 32) g[k] = (float)(-gw[k]);
  __syncwarp();
  bool fail = false;
  for (int k = 0; k < l; ++k) {
    const float d = H[k * l + k];
    if (!(d > 0.f) || !isfinite(d)) fail = true;
    const float dk = d > 0.f ? sqrtf(d) : 1.f;
    __syncwarp();
    if (lane == 0) H[k * l + k] = dk;
    for (int r = k + 1 + lane; r < l; r += 32) H[r * l + k] /= dk;
    __syncwarp();
    for (int r = k + 1 + lane; r < l; r += 32) {
      const float hrk = H[r * l + k];
      for (int c = k + 1; c <= r; ++c) H[r * l + c] -= hrk * H[c * l + k];
    }
    __syncwarp();
  }
  // L y = g (column oriented), then L^T x = y
  for (int r = 0; r < l; ++r) {
    const float yr = g[r] / H[r * l + r];
    __syncwarp();
    if (lane == 0) g[r] = yr;
    for (int i = r + 1 + lane; i < l; i += 32) g[i] -= H[i * l + r] * yr;
    __syncwarp();
  }
  for (int r = l - 1; r >= 0; --r) {
    const float xr = g[r] / H[r * l + r];
    __syncwarp();
    if (lane == 0) g[r] = xr;
    for (int i = lane; i < r; i += 32) g[i] -= H[r * l + i] * xr;
    __syncwarp();
  }
  double dva = 0.0;
  bool finite = true;
  for (int k = lane; k < l; k += 32) {
    P.delta[k] = (double)g[k];
    dva += (double)g[k] * P.Va[k];
    finite = finite && isfinite(g[k]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dva += __shfl_xor_sync(0xffffffffu, dva, o);
  finite = __all_sync(0xffffffffu, finite);
  fail = __any_sync(0xffffffffu, fail) || st->nr_degenerate != 0;
  __syncwarp();
  if (lane == 0) {
    st->nr_degenerate = 0;
    if (fail || !finite) {
      st->nr_ok = 0;
      st->nr_rej += 1;
      st->cur_g = (st->cur_g + 1) % 3;   // keep the Sinkhorn step: g_{k+1} = h
    } else {
      st->nr_ok = 1;
      st->dot_vd_a = dva;
    }
  }
}

// f' = f_k + V Delta (float64 accumulation of float32 V), into the other f buffer.
__global__ void fprime_kernel(const Prob* __restrict__ PP) {
  const Prob& P = *PP;
  const State* st = P.st;
  if (st->done || !st->nr_ok) return;
  const int cf = st->cur_f, l = P.ell;
  // the step V Delta is accumulated in float32 (it is a small correction; the
  // trial pass evaluates exactly the f' stored here)
  __shared__ float d[kMaxK];
  for (int k = threadIdx.x; k < l; k += blockDim.x) d[k] = (float)P.delta[k];
  __syncthreads();
  const double* f = P.f[cf];
  double* fo = P.f[1 - cf];
  const Split so = P.rs[1 - cf];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    const float* Vi = P.V + (size_t)i * l;
    float corr = 0.f;
    for (int k = 0; k < l; ++k) corr = __fmaf_rn(Vi[k], d[k], corr);
    const double v = f[i] + (double)corr;
    fo[i] = v;
    if (P.fA64[0]) P.fA64[1 - cf][i] = v + P.eps * P.loga[i];
    double hi;
    float lo;
    split_grid(v + P.eps * P.loga[i], P.qscale, P.qinv, hi, lo);
    so.A[i] = (float)(hi + (double)P.M);
    so.AL[i] = lo;
    split_grid(v, P.qscale, P.qinv, hi, lo);
    so.K[i] = (float)((double)P.M - hi);
    so.KL[i] = lo;
  }
}

// ---------------------------------------------------------------------------
// Mode computation: one CTA, float32 (the projected p x p problems only need
// a good basis; the float64 Gram sums come in from wgram).
//   inputs  GXX = X^T D_a X, T = Z^T D_a X, c = a^T X   (float64, p x p / p)
//   mode 0 (orthonormalise only, X is the start block):  B = L^{-T},
//           L L^T = GXX - c c^T
//   mode 1 (Rayleigh-Ritz + power step): T = Q Theta Q^T (cyclic Jacobi with
//           the circle ordering, descending Ritz values),
//           residual_k^2 = (Q^T GXX Q)_kk - theta_k^2, then
//           L L^T = Q^T (GXX - c c^T) Q and B = Q L^{-T}.
//   outputs B (p x p float32), theta (p), max residual over the first l.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) eig_small_kernel(int p, int l, int mode,
                                                        const double* __restrict__ GXX,
                                                        const double* __restrict__ T,
                                                        const double* __restrict__ c,
                                                        float* __restrict__ Bout,
                                                        double* __restrict__ theta_out,
                                                        double* __restrict__ resid_out,
                                                        int* __restrict__ fail_out) {
  // A and Q use an odd row stride (pe + 1): the column rotations walk down
  // columns, and an even stride would put many rows in one shared-memory bank
  __shared__ float A[kMaxP * (kMaxP + 1)];
  __shared__ float Q[kMaxP * (kMaxP + 1)];
  __shared__ float G[kMaxP * kMaxP];
  __shared__ float tmp[kMaxP * kMaxP];
  __shared__ float rc[kMaxP], rs[kMaxP], cf[kMaxP], qc[kMaxP];
  __shared__ int pairs[kMaxP];
  __shared__ float th[kMaxP];
  __shared__ int order[kMaxP];
  __shared__ float s_w[16];
  __shared__ int s_stop, s_fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int pe = (p + 1) & ~1;   // padded even size for the circle ordering
  const int ps = pe + 1;         // row stride of A and Q
  for (int e = tid; e < pe * pe; e += nt) {
    const int r = e / pe, q = e - r * pe;
    const bool in = r < p && q < p;
    A[r * ps + q] = (mode == 1 && in) ? (float)(0.5 * (T[r * p + q] + T[q * p + r])) : 0.f;
    Q[r * ps + q] = (r == q) ? 1.f : 0.f;
  }
  for (int k = tid; k < p; k += nt) cf[k] = (float)c[k];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  if (mode == 1) {
    for (int sweep = 0; sweep < 12; ++sweep) {
      float loc = 0.f, dia = 0.f;
      for (int e = tid; e < pe * pe; e += nt) {
        const int r = e / pe, q = e - r * pe;
        const float v = A[r * ps + q];
        if (r != q) loc += v * v;
        else dia += v * v;
      }
      loc = warp_sum_f(loc);
      dia = warp_sum_f(dia);
      if ((tid & 31) == 0) { s_w[tid >> 5] = loc; s_w[8 + (tid >> 5)] = dia; }
      __syncthreads();
      if (tid == 0) {
        float o = 0.f, d = 0.f;
        for (int w = 0; w < (nt >> 5); ++w) { o += s_w[w]; d += s_w[8 + w]; }
        s_stop = (o <= 1e-10f * (d + 1e-30f)) ? 1 : 0;
      }
      __syncthreads();
      if (s_stop) break;
      for (int round = 0; round < pe - 1; ++round) {
        if (tid < pe / 2) {
          const int pa = tid, pb = pe - 1 - tid;
          const int a = pa == 0 ? 0 : 1 + (pa - 1 + round) % (pe - 1);
          const int b = 1 + (pb - 1 + round) % (pe - 1);
          const int k = min(a, b), q = max(a, b);
          pairs[2 * tid] = k;
          pairs[2 * tid + 1] = q;
          const float akq = A[k * ps + q];
          float cth = 1.f, sth = 0.f;
          if (fabsf(akq) > 1e-30f) {
            const float tau = (A[q * ps + q] - A[k * ps + k]) / (2.f * akq);
            const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            cth = rsqrtf(1.f + t * t);
            sth = t * cth;
          }
          rc[tid] = cth;
          rs[tid] = sth;
        }
        __syncthreads();
        for (int e = tid; e < (pe / 2) * pe; e += nt) {     // rows: A <- J^T A
          const int pr = e / pe, col = e - pr * pe;
          const int k = pairs[2 * pr], q = pairs[2 * pr + 1];
          const float cth = rc[pr], sth = rs[pr];
          const float ak = A[k * ps + col], aq = A[q * ps + col];
          A[k * ps + col] = cth * ak - sth * aq;
          A[q * ps + col] = sth * ak + cth * aq;
        }
        __syncthreads();
        for (int e = tid; e < (pe / 2) * pe; e += nt) {     // columns: A <- A J, Q <- Q J
          const int pr = e / pe, row = e - pr * pe;
          const int k = pairs[2 * pr], q = pairs[2 * pr + 1];
          const float cth = rc[pr], sth = rs[pr];
          const float ak = A[row * ps + k], aq = A[row * ps + q];
          A[row * ps + k] = cth * ak - sth * aq;
          A[row * ps + q] = sth * ak + cth * aq;
          const float qk = Q[row * ps + k], qq = Q[row * ps + q];
          Q[row * ps + k] = cth * qk - sth * qq;
          Q[row * ps + q] = sth * qk + cth * qq;
        }
        __syncthreads();
      }
    }
    for (int k = tid; k < p; k += nt) th[k] = A[k * ps + k];
    __syncthreads();
    for (int k = tid; k < p; k += nt) {
      int rank = 0;
      for (int q = 0; q < p; ++q) rank += (th[q] > th[k]) || (th[q] == th[k] && q < k);
      order[rank] = k;
    }
    __syncthreads();
    for (int e = tid; e < p * p; e += nt) {
      const int r = e / p, q = e - r * p;
      tmp[r * p + q] = Q[r * ps + order[q]];
    }
    __syncthreads();
    for (int e = tid; e < p * p; e += nt) Q[e] = tmp[e];
    if (tid < p) theta_out[tid] = (double)th[order[tid]];
    __syncthreads();
  } else {
    for (int e = tid; e < p * p; e += nt) {
      const int r = e / p, q = e - r * p;
      Q[e] = (r == q) ? 1.f : 0.f;
    }
    __syncthreads();
  }
  // G = GXX - c c^T (float), then (mode 1) G <- Q^T G Q
  for (int e = tid; e < p * p; e += nt) {
    const int r = e / p, q = e - r * p;
    G[e] = (float)(GXX[e] - c[r] * c[q]);
  }
  __syncthreads();
  if (mode == 1) {
    for (int e = tid; e < p * p; e += nt) {     // tmp = G Q
      const int r = e / p, q = e - r * p;
      float acc = 0.f;
      for (int k = 0; k < p; ++k) acc = __fmaf_rn(G[r * p + k], Q[k * p + q], acc);
      tmp[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < p * p; e += nt) {     // A = Q^T tmp (stride p)
      const int r = e / p, q = e - r * p;
      float acc = 0.f;
      for (int k = 0; k < p; ++k) acc = __fmaf_rn(Q[k * p + r], tmp[k * p + q], acc);
      A[e] = acc;
    }
    for (int k = tid; k < p; k += nt) {         // (Q^T c)_k
      float acc = 0.f;
      for (int r = 0; r < p; ++r) acc = __fmaf_rn(Q[r * p + k], cf[r], acc);
      qc[k] = acc;
    }
    __syncthreads();
    // residual_k^2 = (Q^T GXX Q)_kk - theta_k^2 = G'_kk + (Q^T c)_k^2 - theta_k^2
    float rmax = 0.f;
    for (int k = tid; k < l && k < p; k += nt) {
      const float t = (float)theta_out[k];
      const float r2 = A[k * p + k] + qc[k] * qc[k] - t * t;
      rmax = fmaxf(rmax, r2 > 0.f ? sqrtf(r2) : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if ((tid & 31) == 0) s_w[tid >> 5] = rmax;
    __syncthreads();
    if (tid == 0) {
      float mx = 0.f;
      for (int w = 0; w < (nt >> 5); ++w) mx = fmaxf(mx, s_w[w]);
      *resid_out = (double)mx;
    }
    for (int e = tid; e < p * p; e += nt) G[e] = A[e];
    __syncthreads();
  }
  // Cholesky of G (lower, in place)
  for (int k = 0; k < p; ++k) {
    const float d = G[k * p + k];
    const float dk = d > 0.f ? sqrtf(d) : 1.f;
    if (tid == 0 && !(d > 0.f)) s_fail = 1;
    __syncthreads();
    if (tid == 0) G[k * p + k] = dk;
    for (int r = k + 1 + tid; r < p; r += nt) G[r * p + k] /= dk;
    __syncthreads();
    for (int e = tid; e < (p - k - 1) * (p - k - 1); e += nt) {
      const int r = k + 1 + e / (p - k - 1), q = k + 1 + e % (p - k - 1);
      if (q <= r) G[r * p + q] -= G[r * p + k] * G[q * p + k];
    }
    __syncthreads();
  }
  // B = Q L^{-T}: row r of B solves  B_r L^T = Q_r  (thread r, in place in tmp)
  for (int e = tid; e < p * p; e += nt) tmp[e] = Q[e];
  __syncthreads();
  for (int r = tid; r < p; r += nt) {
    float* row = tmp + r * p;
    for (int q = 0; q < p; ++q) {
      float acc = row[q];
      for (int k = 0; k < q; ++k) acc -= row[k] * G[q * p + k];
      row[q] = acc / G[q * p + q];
    }
  }
  __syncthreads();
  for (int e = tid; e < p * p; e += nt) Bout[e] = tmp[e];
  if (tid == 0 && fail_out) *fail_out = s_fail;
}

// Z_i <- (X_i - c) B   (len x p, float32), c float64 (deflation of the constant).
// CTA: 64 rows staged in shared memory with B.
__global__ void __launch_bounds__(256) apply_kernel(const float* __restrict__ X,
                                                    const double* __restrict__ c,
                                                    const float* __restrict__ B, int len, int p,
                                                    float* __restrict__ Z) {
  extern __shared__ float sB[];
  float* sX = sB + p * p;   // [64][p]
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) sB[e] = B[e];
  const int r0 = blockIdx.x * 64;
  const int nr = min(64, len - r0);
  for (int e = threadIdx.x; e < 64 * p; e += blockDim.x) {
    const int r = e / p, k = e - r * p;
    sX[e] = r < nr ? X[(size_t)r0 * p + e] - (float)c[k] : 0.f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * p; e += blockDim.x) {
    const int r = e / p, q = e - r * p;
    float s = 0.f;
    for (int k = 0; k < p; ++k) s = __fmaf_rn(sX[r * p + k], sB[k * p + q], s);
    Z[(size_t)(r0 + r) * p + q] = s;
  }
}

// SplitMix64 start block (Steele, Lea & Flood 2014): u = top 53 bits / 2^53,
// entry (i, k) uses counter seed + (i*p + k + 1) * gamma; columns < keep are
// copied from src (n x keep, float32) instead.
__global__ void init_block_kernel(float* __restrict__ Z, int len, int p, unsigned long long seed,
                                  const float* __restrict__ src, int keep) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len * p; e += gridDim.x * blockDim.x) {
    const int i = e / p, k = e - i * p;
    if (k < keep && src) {
      Z[e] = src[(size_t)i * keep + k];
      continue;
    }
    unsigned long long z = seed + (unsigned long long)(e + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= (z >> 31);
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    Z[e] = (float)(2.0 * u - 1.0);
  }
}

// Copy the first l columns of a p-wide block (row-major) into an l-wide array.
__global__ void take_cols_kernel(const float* __restrict__ Z, int len, int p, int l,
                                 float* __restrict__ V) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len * l; e += gridDim.x * blockDim.x) {
    const int i = e / l, k = e - i * l;
    V[e] = Z[(size_t)i * p + k];
  }
}

// d_j = -expm1(L_j) as float64 weights for the gradient reduction.
__global__ void grad_weights_kernel(const Prob* __restrict__ PP, double* __restrict__ d) {
  const Prob& P = *PP;
  if (P.st->done) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.m; j += gridDim.x * blockDim.x)
    d[j] = -(double)expm1f(P.Lcol[j]);
}

}  // namespace eotk
