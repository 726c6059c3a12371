// Small dense algebra on the device for SK-NR(l) (Algorithm 4.1) and the mode
// computation (Sec. 4), plus the O(n l) vector updates.
//
//  * eig_gram_kernel: the fused weighted Gram sums X^T D_w X, Z^T D_w X, X^T w
//    (float32 register blocks, compensated float32 sums across row ranges);
//  * newton_kernel (one CTA): H_V = -(1/eps) [V^T D_a V - W^T D_b^{-1} W]
//    (Eq. d2Q_semi restricted to V_l with D_r ~ D_a, or exact with D_r),
//    grad_V = -sum_j d_j W_j with d_j = 1 - exp((g_j - h_j)/eps) (the semi-dual
//    gradient a - pi(f_k, h) 1 of Eq. dQ_semi projected on V; the row marginals
//    of pi(f_k, g_k) are exactly a after the row half-step), Cholesky of -H_V,
//    Delta = (-H_V)^{-1} grad_V; a failed factorisation rejects the step;
//  * fprime_kernel: f' = f_k + V Delta and its split arrays;
//  * eig_small_kernel (one CTA, float32 Jacobi): Rayleigh-Ritz of the block
//    subspace iteration and the Cholesky-QR transform of the next block;
//  * apply_kernel: Z <- (X - 1 c^T) B.
#include <algorithm>
#include "eot_device.cuh"
#include "eot_internal.h"

namespace eotk {

cudaError_t launch_wtw_reduce(const AccArgs& a, double* WtW, double* gw, cudaStream_t s);

// ---------------------------------------------------------------------------
// Fused weighted Gram sums of the subspace iteration and the Newton set-up:
//   G = X^T D_w X,  T = Z^T D_w X (when Z is given),  c = X^T w.
// eig_gram_kernel: each CTA sums a contiguous range of rows with 4 x 4
// register blocks (float32) into a partial record; eig_gram_reduce_kernel:
// one thread per output element adds the records in range order with a
// compensated float32 sum and writes the float64 result (deterministic).
// ---------------------------------------------------------------------------
constexpr int kEGMaxChunks = 128;
constexpr int kEGRows = 64;      // rows staged in shared memory at a time

__global__ void __launch_bounds__(256) eig_gram_kernel(const float* __restrict__ X,
                                                       const float* __restrict__ Z,
                                                       const double* __restrict__ w, int len,
                                                       int p, float* __restrict__ part,
                                                       const int* __restrict__ skip) {
  pdl_enter();
  if (skip && *skip) return;
  extern __shared__ float sm[];
  float* sX = sm;                         // [kEGRows][p]
  float* sZ = sX + kEGRows * p;           // [kEGRows][p]
  float* sw = sZ + kEGRows * p;           // [kEGRows]
  const int tid = threadIdx.x;
  const int nb = (p + 3) >> 2, nb2 = nb * nb;
  const int ngt = (Z ? 2 : 1) * nb2;               // G and T blocks
  const int nblk = ngt + nb;                       // + c groups
  const int rec = 2 * p * p + p;                   // floats per partial record
  const long long r_beg = (long long)len * blockIdx.x / gridDim.x;
  const long long r_end = (long long)len * (blockIdx.x + 1) / gridDim.x;
  float o[2][4][4];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) o[q][x][y] = 0.f;
  int ua[2][4], va[2][4];                          // clamped column indices of the blocks
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int blk = tid + 256 * q;
    int br = 0, bc = 0;
    if (blk < ngt) {
      const int b = blk >= nb2 ? blk - nb2 : blk;
      br = b / nb;
      bc = b - br * nb;
    } else if (blk < nblk) {
      br = blk - ngt;
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      ua[q][x] = min(4 * br + x, p - 1);
      va[q][x] = min(4 * bc + x, p - 1);
    }
  }
  for (long long r0 = r_beg; r0 < r_end; r0 += kEGRows) {
    const int nr = (int)min((long long)kEGRows, r_end - r0);
    __syncthreads();
    for (int e = tid; e < nr * p; e += 256) {
      sX[e] = X[(size_t)r0 * p + e];
      if (Z) sZ[e] = Z[(size_t)r0 * p + e];
    }
    for (int r = tid; r < nr; r += 256) sw[r] = (float)w[r0 + r];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int blk = tid + 256 * q;
      if (blk >= nblk) continue;
      if (blk < ngt) {
        const float* U = blk >= nb2 ? sZ : sX;
        for (int r = 0; r < nr; ++r) {
          const float wr = sw[r];
          float u[4], v[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            u[x] = wr * U[r * p + ua[q][x]];
            v[x] = sX[r * p + va[q][x]];
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) o[q][x][y] = __fmaf_rn(u[x], v[y], o[q][x][y]);
        }
      } else {
        for (int r = 0; r < nr; ++r) {
          const float wr = sw[r];
#pragma unroll
          for (int x = 0; x < 4; ++x) o[q][0][x] = __fmaf_rn(wr, sX[r * p + ua[q][x]], o[q][0][x]);
        }
      }
    }
  }
  // partial record of this range: [G p*p | T p*p | c p]
  float* my = part + (size_t)blockIdx.x * rec;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int blk = tid + 256 * q;
    if (blk >= nblk) continue;
    if (blk < ngt) {
      const bool isT = blk >= nb2;
      const int b = isT ? blk - nb2 : blk;
      const int br = b / nb, bc = b - br * nb;
      float* dst = my + (isT ? p * p : 0);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int r = 4 * br + x, cc = 4 * bc + y;
          if (r < p && cc < p) dst[r * p + cc] = o[q][x][y];
        }
    } else {
      const int b = blk - ngt;
#pragma unroll
      for (int x = 0; x < 4; ++x)
        if (4 * b + x < p) my[2 * p * p + 4 * b + x] = o[q][0][x];
    }
  }
}

__global__ void __launch_bounds__(64) eig_gram_reduce_kernel(const float* __restrict__ part,
                                                             int nch, int p, int withT,
                                                             double* __restrict__ G,
                                                             double* __restrict__ T,
                                                             double* __restrict__ c,
                                                             const int* __restrict__ skip) {
  pdl_enter();
  if (skip && *skip) return;
  const int rec = 2 * p * p + p;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rec) return;
  const bool isT = e >= p * p && e < 2 * p * p;
  if (isT && !withT) return;
  float sum = 0.f, comp = 0.f;
  for (int k0 = 0; k0 < nch; k0 += 8) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = k0 + k < nch ? __ldg(part + (size_t)(k0 + k) * rec + e) : 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float y = v[k] - comp;
      const float t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    }
  }
  if (e < p * p) G[e] = (double)sum;
  else if (isT) T[e - p * p] = (double)sum;
  else c[e - 2 * p * p] = (double)sum;
}

void launch_eig_gram(const float* X, const float* Z, const double* w, int len, int p,
                     float* part, double* G, double* T, double* c, cudaStream_t s,
                     const int* skip) {
  const int nch = std::max(1, std::min(kEGMaxChunks, (len + kEGRows - 1) / kEGRows));
  const size_t sm = ((size_t)2 * kEGRows * p + kEGRows) * sizeof(float);
  launch_pdl(eig_gram_kernel, dim3(nch), dim3(256), sm, s, X, Z, w, len, p, part, skip);
  const int rec = 2 * p * p + p;
  launch_pdl(eig_gram_reduce_kernel, dim3((rec + 63) / 64), dim3(64), 0, s, part, nch, p, Z ? 1 : 0, G, T, c, skip);
}

// ---------------------------------------------------------------------------
// In-place L1 D L1^T of the symmetric matrix H in shared memory (row stride S,
// lower triangle read), pivots 0..p-1, NB pivots at a time (right-looking,
// outer products, no square roots).  Rows p..rows-1 are right-hand sides that
// ride along as extra rows: their first p entries end as L1^{-1} b.  On
// return H[r][j] = L1_rj D_j (r > j), H[j][j] = D_j, inv[j] = 1 / D_j.  A pivot
// that is not finite or not above `tiny` gets inv 0 (its column then takes no
// part in the later updates) and sets *fail, except that with null_ok a pivot
// of exactly 0 (a zero row and column: a direction that is not there) does
// not count as a failure.
// Every thread factors the NB x NB diagonal block in registers from shared
// memory (no barrier for it); the panel below it and the trailing update take
// one barrier each, NB pivots per pair of barriers instead of one barrier per
// pivot.  Each entry receives the same updates, in the same order and with the
// same products (L1_ru D_u / D_u) x (L1_qu D_u), as in the one-pivot-at-a-time
// elimination.  Called by every thread of the CTA.
// ---------------------------------------------------------------------------
template <int NB>
__device__ void ldlt_blocked(float* H, int S, int p, int rows, float* inv, int* fail, float tiny,
                             bool null_ok) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int NY = nt >> 4, ty = tid >> 4, tx = tid & 15;   // 16-wide tiling of the update
  for (int k0 = 0; k0 < p; k0 += NB) {
    const int nb = min(NB, p - k0), k1 = k0 + nb;
    // (a) the diagonal block: w[j][i] = L1_ji D_i (i < j), d[j] = D_j
    float w[NB][NB], d[NB], di[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      d[j] = 1.f;
      di[j] = 0.f;
#pragma unroll
      for (int i = 0; i < NB; ++i) w[j][i] = 0.f;
      if (j < nb) {
#pragma unroll
        for (int i = 0; i < j; ++i) {
          float t = H[(k0 + j) * S + k0 + i];
#pragma unroll
          for (int u = 0; u < i; ++u) t = __fmaf_rn(-(w[j][u] * di[u]), w[i][u], t);
          w[j][i] = t;
        }
        float t = H[(k0 + j) * S + k0 + j];
#pragma unroll
        for (int u = 0; u < j; ++u) t = __fmaf_rn(-(w[j][u] * di[u]), w[j][u], t);
        d[j] = t;
        const bool ok = t > tiny && isfinite(t);
        di[j] = ok ? 1.f / t : 0.f;
      }
    }
    // (b) the panel below the block: rows k1..rows-1, one thread per row
    for (int r = k1 + tid; r < rows; r += nt) {
      float x[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        x[j] = 0.f;
        if (j < nb) {
          float t = H[r * S + k0 + j];
#pragma unroll
          for (int u = 0; u < j; ++u) t = __fmaf_rn(-(x[u] * di[u]), w[j][u], t);
          x[j] = t;
          H[r * S + k0 + j] = t;
        }
      }
    }
    __syncthreads();
    // (c) the trailing update of rows k1.. and columns k1..min(r, p - 1)
    if (ty < NY) {
      for (int r = k1 + ty; r < rows; r += NY) {
        float hr[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) hr[j] = j < nb ? H[r * S + k0 + j] * di[j] : 0.f;
        const int qe = min(r, p - 1);
        for (int q = k1 + tx; q <= qe; q += 16) {
          float t = H[r * S + q];
#pragma unroll
          for (int j = 0; j < NB; ++j)
            if (j < nb) t = __fmaf_rn(-hr[j], H[q * S + k0 + j], t);
          H[r * S + q] = t;
        }
      }
    }
    // the block's own rows (read by every thread in (a), so written after the
    // barrier) and its pivots
    if (tid == 0) {
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < nb) {
#pragma unroll
          for (int i = 0; i < j; ++i) H[(k0 + j) * S + k0 + i] = w[j][i];
          H[(k0 + j) * S + k0 + j] = d[j];
          inv[k0 + j] = di[j];
          if (di[j] == 0.f && !(null_ok && d[j] == 0.f)) *fail = 1;
        }
      }
    }
    __syncthreads();
  }
}

// Conjugate gradients (Hestenes-Stiefel) for A x = rhs, A the symmetric l x l
// matrix held by its lower triangle in H (row stride kS), rhs in row l of H:
// float32, by the 64 threads of warps 0 and 1 (thread t holds entry t), the
// dot products summed per warp and then over the two warps in order (named
// barrier 1).  Stops at a relative residual of 1e-6 or after 10 l steps;
// returns false when a search direction has non-positive curvature
// p^T A p <= 0 (A is not positive definite along it).  x (shared, l) gets
// the iterate.  Uniform control flow over the 64 threads.
__device__ __forceinline__ void bar64() { asm volatile("bar.sync 1, 64;" ::: "memory"); }
__device__ float cg_dot64(float v, float* red2) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = v;
  bar64();
  const float t = red2[0] + red2[1];
  bar64();
  return t;
}
__device__ bool cg_solve64(const float* H, int kS, int l, float* x, float* sp, float* red2) {
  const int t = threadIdx.x;
  float rv = t < l ? H[l * kS + t] : 0.f, pv = rv, xv = 0.f;
  if (t < 64) sp[t] = pv;
  float rr = cg_dot64(rv * rv, red2);
  const float stop = 1e-12f * fmaxf(rr, 1e-30f);
  bool ok = true;
  for (int it = 0; it < 10 * l && rr > stop; ++it) {
    float ap = 0.f;
    if (t < l)
      for (int c = 0; c < l; ++c)
        ap = __fmaf_rn(c <= t ? H[t * kS + c] : H[c * kS + t], sp[c], ap);
    const float curv = cg_dot64(pv * ap, red2);   // its barriers end the reads of sp
    if (!(curv > 0.f)) {
      ok = false;
      break;
    }
    const float alpha = rr / curv;
    xv = __fmaf_rn(alpha, pv, xv);
    rv = __fmaf_rn(-alpha, ap, rv);
    const float rrn = cg_dot64(rv * rv, red2);
    pv = __fmaf_rn(rrn / rr, pv, rv);
    rr = rrn;
    if (t < 64) sp[t] = pv;
    bar64();
  }
  if (t < l) x[t] = xv;
  bar64();
  return ok;
}

// ---------------------------------------------------------------------------
// Newton step on V (one CTA of 256 threads).  GV = V^T D_a V (or V^T D_r V),
// WtW = sum_j W_j W_j^T / b_j, gw = sum_j d_j W_j (d_j = -expm1(L_j)),
// Va = V^T a.  -eps H_V = GV - WtW is assembled in float64 (the difference
// cancels) and factorised in float32 as L D L^T (outer-product elimination
// without square roots, 8 pivots per pair of barriers: ldlt_blocked; float64
// arithmetic is a small fraction of the float32 rate on this GPU), the forward
// substitution of grad_V = -gw riding along as an extra row;
// Delta = (-H_V)^{-1} grad_V = eps (GV - WtW)^{-1} grad_V.  A pivot that is not
// positive (the restricted Hessian is not negative definite) rejects the step.
// With cg != 0 the system is solved by conjugate gradients (cg_solve64)
// instead of the factorisation; non-positive curvature rejects the step.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) newton_kernel(const Prob* __restrict__ PP,
                                                     const double* __restrict__ WtW,
                                                     const double* __restrict__ gw,
                                                     const double* __restrict__ Dr, int cg) {
  pdl_enter();
  const Prob& P = *PP;
  State* st = P.st;
  if (st->done) return;
  const int l = P.ell;
  if (!EOT_CHECK(l >= 1 && l <= kMaxK, 103)) return;
  const int tid = threadIdx.x, lane = tid & 31;
  const int ty = tid >> 4, tx = tid & 15;          // 16 x 16 tiling of the assembly
  constexpr int kS = kMaxK + 1;                    // odd row stride
  __shared__ float H[(kMaxK + 1) * kS];            // row l: the right-hand side
  __shared__ float g[kMaxK];
  __shared__ float s_inv[kMaxK];   // 1 / D_k
  __shared__ int s_fail;
  const double* __restrict__ G0 = Dr ? Dr : P.GV;
  if (tid == 0) s_fail = 0;
  for (int r = ty; r < l; r += 16)
    for (int c = tx; c <= r; c += 16) {
      const double gv = 0.5 * (G0[r * l + c] + G0[c * l + r]);
      const double wt = 0.5 * (WtW[r * l + c] + WtW[c * l + r]);
      H[r * kS + c] = (float)(gv - wt);
    }
  for (int k = tid; k < l; k += 256) H[l * kS + k] = (float)(-gw[k]);
  __syncthreads();
  if (cg) {
    __shared__ float s_p[64], s_red2[2];
    if (tid >= 64) return;
    const bool ok = cg_solve64(H, kS, l, g, s_p, s_red2);
    if (tid >= 32) return;
    if (lane == 0 && !ok) s_fail = 1;
    __syncwarp();
  } else {
    // elimination (8 pivots per pair of barriers): H[r][k] = L_rk D_k (r > k),
    // H[k][k] = D_k, and row l holds the forward-substituted right-hand side
    ldlt_blocked<8>(H, kS, l, l + 1, s_inv, &s_fail, 0.f, true);
    if (tid >= 32) return;
    for (int k = lane; k < l; k += 32) g[k] = H[l * kS + k];
    __syncwarp();
    // D z = y, then L^T x = z (column oriented, lanes over rows)
    for (int k = lane; k < l; k += 32) g[k] = s_fail ? 0.f : g[k] * s_inv[k];
    __syncwarp();
    for (int k = l - 1; k >= 0; --k) {
      const float xk = g[k];
      for (int i = lane; i < k; i += 32) g[i] = __fmaf_rn(-H[k * kS + i] * s_inv[i], xk, g[i]);
      __syncwarp();
    }
  }
  double dva = 0.0;
  bool finite = true;
  for (int k = lane; k < l; k += 32) {
    const double dk = P.eps * (double)g[k];
    P.delta[k] = dk;
    dva += dk * P.Va[k];
    finite = finite && isfinite(dk);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dva += __shfl_xor_sync(0xffffffffu, dva, o);
  finite = __all_sync(0xffffffffu, finite);
  const bool fail = s_fail != 0 || st->nr_degenerate != 0;
  if (lane == 0) {
    st->nr_degenerate = 0;
    if (fail || !finite) {
      st->nr_ok = 0;
      st->nr_rej += 1;
      trace_trial(P, st, __longlong_as_double(0x7ff8000000000000ll), 0);
      st->cur_g = (st->cur_g + 1) % 3;   // keep the Sinkhorn step: g_{k+1} = h
    } else {
      st->nr_ok = 1;
      st->dot_vd_a = dva;
    }
  }
}

cudaError_t launch_newton(const Prob* dP, const AccArgs& a, double* WtW, double* gw,
                          cudaStream_t s, int cg) {
  cudaError_t e = launch_wtw_reduce(a, WtW, gw, s);
  if (e != cudaSuccess) return e;
  launch_pdl(newton_kernel, dim3(1), dim3(256), 0, s, dP, WtW, gw, nullptr, cg);
  return cudaGetLastError();
}

// f' = f_k + V Delta (float64 accumulation of float32 V), into the other f buffer.
__global__ void fprime_kernel(const Prob* __restrict__ PP) {
  pdl_enter();
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
//   mode 2 (orthonormalise a badly scaled block): as mode 0 with the columns
//           scaled first, Q = diag((GXX - c c^T)_kk^(-1/2)), B = Q L^{-T}.
//   mode 3 (orthonormalise given modes): as mode 0 with the dead-pivot
//           threshold at 1e-5 of the largest pivot instead of 1e-9 (an exactly
//           dependent column keeps a pivot near 1e-6 from the float32 Gram
//           entries; it is dropped instead of becoming amplified noise).
//   outputs B (p x p float32), theta (p), max residual over the first l
//   (mode 1), and (mode 1, when Qout is given) the Ritz rotation Q.  A
//   nonzero *skip makes the launch return at once.
// Launched as one CTA of kMaxP/2 x kMaxP/2 threads (launch_eig_small).
// ---------------------------------------------------------------------------
constexpr int kEH = kMaxP / 2;   // at most kEH x kEH threads: one per pair of pairs
constexpr int kES = kMaxP + 1;   // odd row stride of the shared matrices

// Block-wide sum of two floats; valid in thread 0.
__device__ __forceinline__ void eig_sum2(float& a, float& b, float* red) {
  const int nt = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, w = tid >> 5;
  a = warp_sum_f(a);
  b = warp_sum_f(b);
  if (lane == 0) {
    red[w] = a;
    red[32 + w] = b;
  }
  __syncthreads();
  if (tid == 0) {
    a = b = 0.f;
    for (int k = 0; k < (nt + 31) / 32; ++k) {
      a += red[k];
      b += red[32 + k];
    }
  }
}

// Entry (x, y) of R1 B R2^T for a 2 x 2 block B (b00, b01, b10, b11) and
// rotations R = [[c, -s], [s, c]].
__device__ __forceinline__ float rot_entry(int x, int y, float c1, float s1, float c2, float s2,
                                           float b00, float b01, float b10, float b11) {
  const float u0 = x ? s1 : c1, u1 = x ? c1 : -s1;   // row x of R1
  const float v0 = y ? s2 : c2, v1 = y ? c2 : -s2;   // row y of R2
  return u0 * (b00 * v0 + b01 * v1) + u1 * (b10 * v0 + b11 * v1);
}

// Jacobi rotation annihilating a_kq of the symmetric 2 x 2 problem.
__device__ __forceinline__ void jacobi_rot(float akk, float aqq, float akq, float& cth,
                                           float& sth) {
  cth = 1.f;
  sth = 0.f;
  if (fabsf(akq) > 1e-30f) {
    const float tau = __fdividef(aqq - akk, 2.f * akq);
    const float t = __fdividef(tau >= 0.f ? 1.f : -1.f, fabsf(tau) + sqrtf(1.f + tau * tau));
    cth = rsqrtf(1.f + t * t);
    sth = t * cth;
  }
}

// Out = X Y (or X^T Y) for p x p shared matrices of row stride kES, p <= 2 nx:
// thread (ty, tx) forms the 2 x 2 block of rows ty, ty + nx and columns tx,
// tx + nx.
__device__ __forceinline__ void block2_product(const float* X, const float* Y, float* Out, int p,
                                               int ty, int tx, int nx, bool transX) {
  const int r0 = ty, r1 = ty + nx, q0 = tx, q1 = tx + nx;
  if (r0 >= p || q0 >= p) return;
  const bool vr = r1 < p, vq = q1 < p;
  float a00 = 0.f, a01 = 0.f, a10 = 0.f, a11 = 0.f;
  for (int k = 0; k < p; ++k) {
    const float x0 = transX ? X[k * kES + r0] : X[r0 * kES + k];
    const float x1 = vr ? (transX ? X[k * kES + r1] : X[r1 * kES + k]) : 0.f;
    const float y0 = Y[k * kES + q0];
    const float y1 = vq ? Y[k * kES + q1] : 0.f;
    a00 = __fmaf_rn(x0, y0, a00);
    a01 = __fmaf_rn(x0, y1, a01);
    a10 = __fmaf_rn(x1, y0, a10);
    a11 = __fmaf_rn(x1, y1, a11);
  }
  Out[r0 * kES + q0] = a00;
  if (vq) Out[r0 * kES + q1] = a01;
  if (vr) Out[r1 * kES + q0] = a10;
  if (vr && vq) Out[r1 * kES + q1] = a11;
}

__global__ void __launch_bounds__(kEH * kEH) eig_small_kernel(int p, int l, int mode,
                                                              const double* __restrict__ GXX,
                                                              const double* __restrict__ T,
                                                              const double* __restrict__ c,
                                                              float* __restrict__ Bout,
                                                              double* __restrict__ theta_out,
                                                              double* __restrict__ resid_out,
                                                              int* __restrict__ fail_out,
                                                              float* __restrict__ Qout,
                                                              const int* __restrict__ skip) {
  pdl_enter();
  if (skip && *skip) return;
  if (!EOT_CHECK(p >= 1 && p <= kMaxP && l <= p && 2 * (int)blockDim.x >= p, 104)) return;
  __shared__ float A0[kMaxP * kES];
  __shared__ float Q[kMaxP * kES];
  __shared__ __align__(16) float G[kMaxP * kES];
  __shared__ float W[kMaxP * kES];        // scratch; the second Jacobi buffer
  __shared__ float rc[2][kEH], rs[2][kEH], sq[kMaxP];
  __shared__ int pk[2][kEH], pq[2][kEH];
  __shared__ float th[kMaxP], cf[kMaxP], qc[kMaxP];
  __shared__ int order[kMaxP];
  __shared__ float red[64];
  __shared__ int s_stop, s_fail;
  const int nx = blockDim.x;              // blockDim = (nx, nx), nx >= half
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * nx + tx, nt = nx * nx;
  const int pe = (p + 1) & ~1;            // padded even size for the circle ordering
  const int half = pe / 2, nr = pe - 1;   // pairs per round, rounds per sweep
  float* A = A0;
  for (int r = ty; r < pe; r += nx)
    for (int q = tx; q < pe; q += nx) {
      const bool in = r < p && q < p;
      A[r * kES + q] = (mode == 1 && in) ? (float)(0.5 * (T[r * p + q] + T[q * p + r])) : 0.f;
      Q[r * kES + q] = (r == q) ? 1.f : 0.f;
    }
  for (int k = tid; k < p; k += nt) cf[k] = (float)c[k];
  // circle ordering: index 0 fixed, the others rotate by one place per round;
  // pair (k, q), k < q, of slot t in round r
  auto pair_of = [&](int r, int t, int& k, int& q) {
    const int pa = t, pb = pe - 1 - t;
    const int a = pa == 0 ? 0 : 1 + (pa - 1 + r) % nr;
    const int b = 1 + (pb - 1 + r) % nr;
    k = min(a, b);
    q = max(a, b);
  };
  // Table of the Jacobi rounds (in G, unused until the Jacobi ends): for round
  // r and slot t of round r + 1 (round 0 after the last), its pair (k, q) and
  // where k and q sit in round r: slots ta, tb with pairs (ka, qa), (kb, qb)
  // and sides xa, xb.  Packed: k | q << 6 | ka << 12 | qa << 18 | xa << 24 |
  // xb << 25, and kb | qb << 6 | ta << 12 | tb << 17.
  uint2* nxt = reinterpret_cast<uint2*>(G);
  // slot of index idx in round r (inverse of pair_of): index 0 sits in slot 0;
  // any other index sits at position pos = 1 + (idx - 1 - r mod nr) of the
  // rotating ring, on the first side of slot pos if pos < half, else on the
  // second side of slot pe - 1 - pos
  auto slot_of = [&](int r, int idx, int& t, int& x, int& k2, int& q2) {
    if (idx == 0) {
      t = 0;
    } else {
      const int pos = 1 + ((idx - 1 - r) % nr + nr) % nr;
      t = pos <= half - 1 ? pos : pe - 1 - pos;
    }
    pair_of(r, t, k2, q2);
    x = q2 == idx;
  };
  if (mode == 1) {
    for (int e = tid; e < nr * half; e += nt) {
      const int r = e / half, t = e - r * half;
      int k, q;
      pair_of(r + 1 < nr ? r + 1 : 0, t, k, q);
      int ta, tb, xa, xb, ka, qa, kb, qb;
      slot_of(r, k, ta, xa, ka, qa);
      slot_of(r, q, tb, xb, kb, qb);
      nxt[e] = make_uint2((unsigned)(k | (q << 6) | (ka << 12) | (qa << 18) | (xa << 24) | (xb << 25)),
                          (unsigned)(kb | (qb << 6) | (ta << 12) | (tb << 17)));
    }
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  if (mode == 1) {
    // cyclic Jacobi: in each round the pe/2 disjoint pairs rotate at once;
    // thread (ty, tx) maps the 2 x 2 block of pairs (ty, tx) from A to the
    // other buffer (A' = R A R^T), applies the rotations of pair tx to rows ty
    // and ty + half of Q, and (ty == 0) forms the rotation of slot tx of the
    // next round from the current values: one barrier per round
    float* An = W;
    if (ty == 0 && tx < half) {
      int k, q;
      pair_of(0, tx, k, q);
      pk[0][tx] = k;
      pq[0][tx] = q;
      jacobi_rot(A[k * kES + k], A[q * kES + q], A[k * kES + q], rc[0][tx], rs[0][tx]);
    }
    __syncthreads();
    int cur = 0;
    for (int sweep = 0; sweep < 12; ++sweep) {
      float loc = 0.f, dia = 0.f;
      for (int r = ty; r < pe; r += nx)
        for (int q = tx; q < pe; q += nx) {
          const float v = A[r * kES + q];
          if (r != q) loc += v * v;
          else dia += v * v;
        }
      eig_sum2(loc, dia, red);
      // off-diagonal below 1e-4 of the diagonal (Frobenius): the Ritz
      // vectors then carry errors far below the subspace iteration's residual
      // tolerance, and the next iteration refines them anyway
      if (tid == 0) s_stop = (loc <= 1e-8f * (dia + 1e-30f)) ? 1 : 0;
      __syncthreads();
      if (s_stop) break;
      for (int round = 0; round < nr; ++round) {
        if (ty < half && tx < half) {
          const int k1 = pk[cur][ty], q1 = pq[cur][ty], k2 = pk[cur][tx], q2 = pq[cur][tx];
          const float c1 = rc[cur][ty], s1 = rs[cur][ty], c2 = rc[cur][tx], s2 = rs[cur][tx];
          const float a = A[k1 * kES + k2], b = A[k1 * kES + q2];
          const float e = A[q1 * kES + k2], d = A[q1 * kES + q2];
          const float u11 = c1 * a - s1 * e, u12 = c1 * b - s1 * d;
          const float u21 = s1 * a + c1 * e, u22 = s1 * b + c1 * d;
          An[k1 * kES + k2] = u11 * c2 - u12 * s2;
          An[k1 * kES + q2] = u11 * s2 + u12 * c2;
          An[q1 * kES + k2] = u21 * c2 - u22 * s2;
          An[q1 * kES + q2] = u21 * s2 + u22 * c2;
        }
        if (tx < half) {
          const int k = pk[cur][tx], q = pq[cur][tx];
          const float cth = rc[cur][tx], sth = rs[cur][tx];
          for (int r = ty; r < pe; r += nx) {
            const float qk = Q[r * kES + k], qq = Q[r * kES + q];
            Q[r * kES + k] = cth * qk - sth * qq;
            Q[r * kES + q] = sth * qk + cth * qq;
          }
        }
        if (ty == 0 && tx < half) {
          // slot tx of the next round (round 0 of the next sweep after the last)
          const uint2 tb2 = nxt[round * half + tx];
          const int k = tb2.x & 63, q = (tb2.x >> 6) & 63, ka = (tb2.x >> 12) & 63;
          const int qa = (tb2.x >> 18) & 63, xa = (tb2.x >> 24) & 1, xb = (tb2.x >> 25) & 1;
          const int kb = tb2.y & 63, qb = (tb2.y >> 6) & 63, ta = (tb2.y >> 12) & 31;
          const int tb = (tb2.y >> 17) & 31;
          const float ca = rc[cur][ta], sa = rs[cur][ta], cb = rc[cur][tb], sb = rs[cur][tb];
          const float akk = rot_entry(xa, xa, ca, sa, ca, sa, A[ka * kES + ka], A[ka * kES + qa],
                                      A[qa * kES + ka], A[qa * kES + qa]);
          const float aqq = rot_entry(xb, xb, cb, sb, cb, sb, A[kb * kES + kb], A[kb * kES + qb],
                                      A[qb * kES + kb], A[qb * kES + qb]);
          const float akq = rot_entry(xa, xb, ca, sa, cb, sb, A[ka * kES + kb], A[ka * kES + qb],
                                      A[qa * kES + kb], A[qa * kES + qb]);
          pk[cur ^ 1][tx] = k;
          pq[cur ^ 1][tx] = q;
          jacobi_rot(akk, aqq, akq, rc[cur ^ 1][tx], rs[cur ^ 1][tx]);
        }
        __syncthreads();
        float* t2 = A;
        A = An;
        An = t2;
        cur ^= 1;
      }
    }
    // descending order of the Ritz values by a strict total order (a value
    // that is not a number sorts last, ties by index), so that the ranks are
    // always a permutation of 0..p-1 and every order[] entry is written
    for (int k = tid; k < p; k += nt) {
      const float v = A[k * kES + k];
      th[k] = v == v ? v : -INFINITY;
      if (v != v) s_fail = 1;
    }
    __syncthreads();
    for (int k = tid; k < p; k += nt) {
      int rank = 0;
      for (int q = 0; q < p; ++q) rank += (th[q] > th[k]) || (th[q] == th[k] && q < k);
      order[rank] = k;
    }
    __syncthreads();
    for (int r = ty; r < p; r += nx)      // G = Q with the columns in descending order
      for (int q = tx; q < p; q += nx)
        G[r * kES + q] = EOT_CHECK(order[q] >= 0 && order[q] < p, 101) ? Q[r * kES + order[q]] : 0.f;
    if (tid < p && EOT_CHECK(order[tid] >= 0 && order[tid] < p, 102))
      theta_out[tid] = (double)th[order[tid]];
    __syncthreads();
    for (int r = ty; r < p; r += nx)
      for (int q = tx; q < p; q += nx) {
        Q[r * kES + q] = G[r * kES + q];
        if (Qout) Qout[r * p + q] = G[r * kES + q];   // the Ritz rotation, for the filter
      }
  } else {
    for (int r = ty; r < p; r += nx)
      for (int q = tx; q < p; q += nx) Q[r * kES + q] = (r == q) ? 1.f : 0.f;
  }
  __syncthreads();
  A = A0;
  // G = GXX - c c^T (float), then (modes 1, 2) G <- Q^T G Q
  for (int r = ty; r < p; r += nx)
    for (int q = tx; q < p; q += nx) G[r * kES + q] = (float)(GXX[r * p + q] - c[r] * c[q]);
  __syncthreads();
  if (mode == 2) {
    // column scaling Q = diag(G_kk^(-1/2)): the block's columns may differ in
    // scale by orders of magnitude (a filtered block), which the Cholesky
    // factor of the scaled Gram matrix does not inherit
    for (int r = ty; r < p; r += nx)
      for (int q = tx; q < p; q += nx)
        Q[r * kES + q] = (r == q) ? rsqrtf(fmaxf(G[r * kES + r], 1e-30f)) : 0.f;
    __syncthreads();
  }
  if (mode == 1 || mode == 2) {
    // W = G Q: thread (ty, tx) forms rows ty, ty + nx and columns tx, tx + nx
    // (p <= 2 nx), each loaded value used twice
    block2_product(G, Q, W, p, ty, tx, nx, false);
    if (ty == 0)                          // (Q^T c)_k
      for (int k = tx; k < p; k += nx) {
        float acc = 0.f;
        for (int r = 0; r < p; ++r) acc = __fmaf_rn(Q[r * kES + k], cf[r], acc);
        qc[k] = acc;
      }
    __syncthreads();
    block2_product(Q, W, A, p, ty, tx, nx, true);   // A = Q^T W
    __syncthreads();
    // residual_k^2 = (Q^T GXX Q)_kk - theta_k^2 = G'_kk + (Q^T c)_k^2 - theta_k^2
    float rmax = 0.f;
    for (int k = tid; mode == 1 && k < l && k < p; k += nt) {
      const float t = (float)theta_out[k];
      const float r2 = A[k * kES + k] + qc[k] * qc[k] - t * t;
      rmax = fmaxf(rmax, r2 > 0.f ? sqrtf(r2) : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if ((tid & 31) == 0) red[tid >> 5] = rmax;
    __syncthreads();
    if (tid == 0 && mode == 1) {
      float mx = 0.f;
      for (int w = 0; w < (nt + 31) / 32; ++w) mx = fmaxf(mx, red[w]);
      *resid_out = (double)mx;
    }
    for (int r = ty; r < p; r += nx)
      for (int q = tx; q < p; q += nx) G[r * kES + q] = A[r * kES + q];
    __syncthreads();
  }
  // G = L1 D L1^T (8 pivots per pair of barriers; th: scratch for 1 / D,
  // the Ritz values are written out); L = L1 D^(1/2).  A pivot below 1e-9 of
  // the largest diagonal entry (the block has lost rank: at large eps only a
  // few rho_k^2 are not negligible) marks its column dead: the column becomes
  // exactly zero (sq = 0) instead of amplified rounding noise, which would
  // overflow in the next products.
  if (tid == 0) {
    float mx = 0.f;
    for (int k = 0; k < p; ++k) mx = fmaxf(mx, G[k * kES + k]);
    red[0] = fmaxf((mode == 3 ? 1e-5f : 1e-9f) * mx, 1e-30f);
  }
  __syncthreads();
  const float tiny = red[0];
  __syncthreads();
  ldlt_blocked<8>(G, kES, p, p, th, &s_fail, tiny, false);
  for (int k = tid; k < p; k += nt) {
    const float dk = G[k * kES + k];
    sq[k] = th[k] > 0.f ? rsqrtf(dk) : 0.f;   // 1 / L_kk; 0: dead column
  }
  __syncthreads();
  // L below the diagonal: L_cq = G_cq / sqrt(D_q) (one product per element)
  for (int r = ty; r < p; r += nx)
    for (int q = tx; q < r; q += nx) G[r * kES + q] *= sq[q];
  for (int r = ty; r < p; r += nx)        // W = Q (right-hand sides)
    for (int q = tx; q < p; q += nx) W[r * kES + q] = Q[r * kES + q];
  __syncthreads();
  // B L^T = Q by blocks of 8 columns, B_rq = W_rq sq_q: (a) one thread per
  // row finishes the block's columns (updates from the block's earlier
  // columns), (b) the later columns receive the block's updates; every entry
  // gets its updates in increasing column order, as column by column
  {
    const int NY = nt >> 4, y16 = tid >> 4, x16 = tid & 15;
    for (int c0 = 0; c0 < p; c0 += 8) {
      const int nb = min(8, p - c0), c1 = c0 + nb;
      for (int r = tid; r < p; r += nt) {
        float b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          b[j] = 0.f;
          if (j < nb) {
            float t = W[r * kES + c0 + j];
#pragma unroll
            for (int u = 0; u < j; ++u) t = __fmaf_rn(-b[u], G[(c0 + j) * kES + c0 + u], t);
            W[r * kES + c0 + j] = t;
            b[j] = t * sq[c0 + j];
          }
        }
      }
      __syncthreads();
      if (y16 < NY) {
        for (int r = y16; r < p; r += NY) {
          float b[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) b[j] = j < nb ? W[r * kES + c0 + j] * sq[c0 + j] : 0.f;
          for (int cc = c1 + x16; cc < p; cc += 16) {
            float t = W[r * kES + cc];
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (j < nb) t = __fmaf_rn(-b[j], G[cc * kES + c0 + j], t);
            W[r * kES + cc] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int r = ty; r < p; r += nx)
    for (int q = tx; q < p; q += nx) Bout[r * p + q] = W[r * kES + q] * sq[q];
  if (tid == 0 && fail_out) *fail_out = s_fail;
}

void launch_eig_small(int p, int l, int mode, const double* GXX, const double* T,
                      const double* c, float* B, double* theta, double* resid, int* fail,
                      cudaStream_t s, float* Qout, const int* skip) {
  const int half = std::max(4, ((p + 1) & ~1) / 2);   // one thread per pair of pairs
  launch_pdl(eig_small_kernel, dim3(1), dim3(dim3(half, half)), 0, s, p, l, mode, GXX, T, c, B, theta, resid, fail,
                                                  Qout, skip);
}

// Z_i <- (X_i - c) B   (len x p, float32), c float64 (deflation of the constant).
// CTA: 64 rows staged in shared memory with B.
__global__ void __launch_bounds__(256) apply_kernel(const float* __restrict__ X,
                                                    const double* __restrict__ c,
                                                    const float* __restrict__ B, int len, int p,
                                                    float* __restrict__ Z,
                                                    const int* __restrict__ skip) {
  pdl_enter();
  if (skip && *skip) return;
  if (!EOT_CHECK(p >= 1 && p <= kMaxP && (unsigned)(p * p + 64 * p) * 4u <= dyn_smem_bytes(), 105))
    return;
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

// ---------------------------------------------------------------------------
// Chebyshev-filtered subspace iteration (Sec. 3: the rho^2 cluster near 1 slows
// the plain power method; Sec. 4 asks for an efficient power method).  Between
// two Rayleigh-Ritz steps the Ritz vectors Zr = Z Q are multiplied by the
// Chebyshev polynomial T_d((M - c)/e) with [c - e, c + e] = [0, cut] covering
// the spectrum below the block's smallest Ritz value theta_{p-1} (cut is at
// least 1e-6 theta_0): the part of the spectrum below it stays bounded while
// the wanted eigenvalues grow like cosh(d arccosh x).  The three-term
// recurrence is the scaled one of Zhou and Saad (2007), which divides step k
// by T_k at theta_0 so that the leading components stay of order one in
// float32 (the same span as the unscaled recurrence):
//   sigma_1 = e / (theta_0 - c),  Y_1 = (sigma_1 / e) (M - c) Y_0,
//   sigma_k = 1 / (2 / sigma_1 - sigma_{k-1}),
//   Y_k = (2 sigma_k / e) (M - c) Y_{k-1} - sigma_{k-1} sigma_k Y_{k-2}.
// Every product M Y is deflated of the constant mode (Y - 1 a^T Y).  sig holds
// c, e, sigma_1 and sigma_k at sig[4 + k].  A nonzero *skip (the mode loop
// has converged) makes each step's launches return at once.
// ---------------------------------------------------------------------------
static_assert(kChebSigDoubles >= 5 + kMaxChebDegree, "filter state");

// The Ritz pairs of a Rayleigh-Ritz step, z_k = (Z Q)_k and M z_k = ((X - 1 c^T)
// Q)_k (X = M Z), and the a-norms of their residuals r_k = M z_k - theta_k z_k,
// k < l, formed from the residual vectors themselves (the Gram-matrix identity
// |r_k|^2 = |M z_k|^2 - theta_k^2 cancels to a float32 floor near 1e-3): per
// CTA (16-row tiles, grid-stride) thread (group g, column q) adds
// a_i r_iq^2 over its rows in a fixed order into part[b][q]; the last CTA to
// arrive adds the CTAs' partials in a fixed order and writes max_k |r_k|_a to
// *resid (NaN if any is not a number), then re-arms the counter.  With Y0, Y1
// given it also starts the Chebyshev filter: Y_0 = Z Q, Y_1 = (sigma_1 / e)
// (M Z Q - c Z Q), and writes the filter's scalars into sig.
constexpr int kRitzRows = 16;
__global__ void __launch_bounds__(256) ritz_kernel(const float* __restrict__ Z,
                                                   const float* __restrict__ X,
                                                   const double* __restrict__ cx,
                                                   const float* __restrict__ Q,
                                                   const double* __restrict__ theta,
                                                   const double* __restrict__ a, int len, int p,
                                                   int l, float* __restrict__ part,
                                                   unsigned* __restrict__ cnt,
                                                   double* __restrict__ resid,
                                                   float* __restrict__ Y0, float* __restrict__ Y1,
                                                   double* __restrict__ sig) {
  pdl_enter();
  if (!EOT_CHECK(p >= 1 && p <= kMaxP && l <= p &&
                     (unsigned)(p * p + 2 * kRitzRows * p) * 4u <= dyn_smem_bytes(), 106))
    return;
  extern __shared__ float sQ[];
  float* sZ = sQ + p * p;            // [16][p]
  float* sX = sZ + kRitzRows * p;    // [16][p]
  __shared__ float red[4][64];
  __shared__ double r2[64];
  __shared__ int s_last;
  const int q = threadIdx.x & 63, g = threadIdx.x >> 6;   // column, row group
  double cs = 0.0, e = 1.0, s1 = 1.0;
  if (Y0) {
    const double t0 = theta[0];
    const double cut = fmax(theta[p - 1], 1e-6 * t0);
    cs = 0.5 * cut;
    e = 0.5 * cut;
    if (!(t0 > 0.0) || !(e > 0.0)) {   // no spectrum to separate: a plain power step
      cs = 0.0;
      e = 1.0;
    }
    s1 = (t0 > cs) ? e / (t0 - cs) : 1.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sig[0] = cs;
      sig[1] = e;
      sig[2] = s1;
      sig[5] = s1;
    }
  }
  const float f1 = (float)(s1 / e), fc = (float)cs;
  const float th = q < l ? (float)theta[q] : 0.f;
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) sQ[i] = Q[i];
  float acc = 0.f;
  const int ntiles = (len + kRitzRows - 1) / kRitzRows;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r0 = t * kRitzRows, nr = min(kRitzRows, len - r0);
    __syncthreads();   // the previous tile's rows are read
    for (int i = threadIdx.x; i < kRitzRows * p; i += blockDim.x) {
      const int r = i / p, k = i - r * p;
      sZ[i] = r < nr ? Z[(size_t)r0 * p + i] : 0.f;
      sX[i] = r < nr ? X[(size_t)r0 * p + i] - (float)cx[k] : 0.f;
    }
    __syncthreads();
    if (q < p) {
      for (int r = g; r < nr; r += 4) {
        // four independent partial sums per product (short dependency chains)
        float za[4] = {0.f, 0.f, 0.f, 0.f}, xa[4] = {0.f, 0.f, 0.f, 0.f};
        int k = 0;
        for (; k + 4 <= p; k += 4) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float qv = sQ[(k + u) * p + q];
            za[u] = __fmaf_rn(sZ[r * p + k + u], qv, za[u]);
            xa[u] = __fmaf_rn(sX[r * p + k + u], qv, xa[u]);
          }
        }
        for (; k < p; ++k) {
          const float qv = sQ[k * p + q];
          za[0] = __fmaf_rn(sZ[r * p + k], qv, za[0]);
          xa[0] = __fmaf_rn(sX[r * p + k], qv, xa[0]);
        }
        const float z = (za[0] + za[1]) + (za[2] + za[3]);
        const float x = (xa[0] + xa[1]) + (xa[2] + xa[3]);
        if (q < l) {
          const float res = __fmaf_rn(-th, z, x);
          acc = __fmaf_rn((float)a[r0 + r] * res, res, acc);
        }
        if (Y0) {
          Y0[(size_t)(r0 + r) * p + q] = z;
          Y1[(size_t)(r0 + r) * p + q] = f1 * __fmaf_rn(-fc, z, x);
        }
      }
    }
  }
  red[g][q] = acc;
  __syncthreads();
  if (threadIdx.x < l) part[(size_t)blockIdx.x * l + threadIdx.x] =
      (red[0][threadIdx.x] + red[1][threadIdx.x]) + (red[2][threadIdx.x] + red[3][threadIdx.x]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last CTA: column q, chunk g of the partials, eight loads in flight
  const int nch = gridDim.x;
  double t = 0.0;
  if (q < l) {
    for (int b0 = g * 8; b0 < nch; b0 += 32) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = b0 + u < nch ? __ldcg(part + (size_t)(b0 + u) * l + q) : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) t += (double)v[u];
    }
  }
  if (g == 0) r2[q] = 0.0;
  __syncthreads();
  for (int gg = 0; gg < 4; ++gg) {   // fixed order over the chunks
    if (g == gg && q < l) r2[q] += t;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < l; ++k) mx = (r2[k] == r2[k] && mx == mx) ? fmax(mx, r2[k]) : NAN;
    *resid = sqrt(mx);   // NaN if any residual was (the loop then stops as failed)
    *cnt = 0u;
  }
}

// Partial sums a^T X over row ranges: part[b][k] for CTA b (8 warps over rows,
// lanes over columns, fixed order).
__global__ void __launch_bounds__(256) wsum_part_kernel(const float* __restrict__ X,
                                                        const double* __restrict__ a, int len,
                                                        int p, float* __restrict__ part,
                                                        const int* __restrict__ skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ float red[8][kMaxP];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r_beg = (int)((long long)len * blockIdx.x / gridDim.x);
  const int r_end = (int)((long long)len * (blockIdx.x + 1) / gridDim.x);
  float s0 = 0.f, s1 = 0.f;
  for (int i = r_beg + w; i < r_end; i += 8) {
    const float ai = (float)a[i];
    if (lane < p) s0 = __fmaf_rn(ai, X[(size_t)i * p + lane], s0);
    if (lane + 32 < p) s1 = __fmaf_rn(ai, X[(size_t)i * p + lane + 32], s1);
  }
  if (lane < p) red[w][lane] = s0;
  if (lane + 32 < p) red[w][lane + 32] = s1;
  __syncthreads();
  for (int k = threadIdx.x; k < p; k += blockDim.x) {
    float t = 0.f;
    for (int v = 0; v < 8; ++v) t += red[v][k];
    part[(size_t)blockIdx.x * p + k] = t;
  }
}

// Step k of the recurrence: Yp <- (2 sigma_k / e) ((X - 1 c^T) - c Yc) -
// sigma_{k-1} sigma_k Yp, X = M Yc, c = a^T X from the nch partials.
__global__ void __launch_bounds__(256) cheb_step_kernel(const float* __restrict__ X,
                                                        const float* __restrict__ part, int nch,
                                                        const float* __restrict__ Yc,
                                                        float* __restrict__ Yp, int len, int p,
                                                        int k, double* __restrict__ sig,
                                                        const int* __restrict__ skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ float cx[kMaxP];
  for (int q = threadIdx.x; q < p; q += blockDim.x) {
    double t = 0.0;
    for (int b0 = 0; b0 < nch; b0 += 8) {   // eight loads in flight, then the adds
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = b0 + u < nch ? part[(size_t)(b0 + u) * p + q] : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) t += (double)v[u];
    }
    cx[q] = (float)t;
  }
  const double cs = sig[0], e = sig[1], s1 = sig[2], sp = sig[4 + k - 1];
  const double sk = 1.0 / (2.0 / s1 - sp);
  if (blockIdx.x == 0 && threadIdx.x == 0) sig[4 + k] = sk;
  __syncthreads();
  const float fa = (float)(2.0 * sk / e), fb = (float)(sp * sk), fc = (float)cs;
  const long long total = (long long)len * p;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i % p);
    const float mx = X[i] - cx[q];
    Yp[i] = __fmaf_rn(fa, __fmaf_rn(-fc, Yc[i], mx), -fb * Yp[i]);
  }
}

// The Ritz residuals (and, with Y0 given, the filter's start) into *resid;
// part: at least 256 x l floats of scratch, cnt: an arrival counter at 0.
void launch_ritz(const float* Z, const float* X, const double* cx, const float* Q,
                 const double* theta, const double* a, int len, int p, int l, float* part,
                 unsigned* cnt, float* Y0, float* Y1, double* sig, double* resid, int nsm,
                 cudaStream_t s) {
  const int ntiles = (len + kRitzRows - 1) / kRitzRows;
  const int grid = std::max(1, std::min(ntiles, std::min(256, 2 * nsm)));
  const size_t sm = ((size_t)p * p + 2 * kRitzRows * p) * sizeof(float);
  launch_pdl(ritz_kernel, dim3(grid), dim3(256), sm, s, Z, X, cx, Q, theta, a, len, p, l, part, cnt, resid, Y0, Y1,
                                    sig);
}

// One filter step after the product X = M Yc: the deflation sums and the
// recurrence (part: at least 128 x p floats of scratch).
void launch_cheb_step(const float* X, const double* a, const float* Yc, float* Yp, int len, int p,
                      int k, double* sig, float* part, int nsm, const int* skip, cudaStream_t s) {
  const int nch = std::max(1, std::min(128, (len + 31) / 32));
  launch_pdl(wsum_part_kernel, dim3(nch), dim3(256), 0, s, X, a, len, p, part, skip);
  const long long total = (long long)len * p;
  const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 4LL * nsm));
  launch_pdl(cheb_step_kernel, dim3(grid), dim3(256), 0, s, X, part, nch, Yc, Yp, len, p, k, sig, skip);
}

// SplitMix64 start block (Steele, Lea & Flood 2014): u = top 53 bits / 2^53,
// entry (i, k) uses counter seed + (i*p + k + 1) * gamma; columns < keep are
// copied from src (n x keep, float32) instead, except (redraw_zero != 0) its
// zero entries, so that a dead (zero) column of earlier modes is drawn anew.
__global__ void init_block_kernel(float* __restrict__ Z, int len, int p, unsigned long long seed,
                                  const float* __restrict__ src, int keep, int redraw_zero) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len * p; e += gridDim.x * blockDim.x) {
    const int i = e / p, k = e - i * p;
    if (k < keep && src) {
      const float v = src[(size_t)i * keep + k];
      if (v != 0.f || !redraw_zero) {
        Z[e] = v;
        continue;
      }
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

EOT_DEBUG_UNIT(small)

}  // namespace eotk
