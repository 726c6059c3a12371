// Internal structures shared by the kernels and the host driver.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <utility>

namespace eotk {

// Launch with programmatic stream serialization: the kernel may be launched
// while the preceding kernel of the stream is still running (its launch and
// CTA start-up overlap that kernel's tail); the kernel calls pdl_enter (or
// pdl_wait) before touching anything the preceding kernels write.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Column pass tile: 128 output columns per CTA (32 lanes x 4), 8 warps over rows.
constexpr int kColTile = 128;
// Row pass tile: 8 warps x 4 rows = 32 output rows per CTA.
constexpr int kRowsPerWarp = 4;
constexpr int kRowTile = 8 * kRowsPerWarp;
constexpr int kThreads = 256;
// Widest mode block handled by the accumulating passes.
constexpr int kMaxK = 64;
// Widest block of the subspace iteration (modes + oversampling).
constexpr int kMaxP = 48;
// Chebyshev filter of the subspace iteration: highest degree, and the doubles
// of its state (c, e, sigma_1, sigma_k at 4 + k).
constexpr int kMaxChebDegree = 8;
constexpr int kChebSigDoubles = 16;

// What the grid-wide final step of a pass does with its reductions.
enum PassMode : int {
  MODE_PLAIN = 0,     // standalone transform: write outputs only
  MODE_SK_COL = 1,    // Sinkhorn column pass: convergence test, advance g
  MODE_SK_ROW = 2,    // Sinkhorn / SK-NR row pass
  MODE_S4_F32 = 3,    // SK-NR column pass at f_k (float32 path, tensor-core kernel)
  MODE_TRIAL = 4,     // SK-NR trial column pass at f': accept / reject
  MODE_EVAL = 5,      // marginal evaluation only (no potential update)
  MODE_G_INIT = 6,    // first column transform of a level (Alg. 4.1 line 3, k = 1)
  MODE_S4 = 7         // float64 SK-NR column pass (h, W)
};

// What a coupling-product pass computes (AccArgs::mode): the column product
// Op(pi)^T Z, the fused SK-NR column pass S4, the row product Op(pi) Z.
enum AccMode : int { ACC_KCOL = 0, ACC_S4 = 1, ACC_KROW = 2 };

// One record of the per-solve iteration trace (the layout of eot_trace_rec):
// the level's eps, the L1 test at f_k and Q_semi(f_k) of iteration `iter`,
// and the Newton trial's dq with its outcome (1 accepted, 0 rejected or not
// solvable, -1 no trial: plain Sinkhorn, or the level stopped at the test).
struct TraceRec {
  double eps, l1, q_semi, dq;
  int iter, accepted;
};

// Device-resident solver state (one per problem).
struct State {
  int iter;        // Algorithm 4.1 iterations done at the current level
  int done;        // 0 running, 1 converged, 2 max_iter, 3 numeric error,
                   // 4 loop body cap, 5 a grid-barrier wait gave up,
                   // 6 the L1 error stalled (see stop_code)
  int cur_f;       // index of the current f buffer (0/1)
  int cur_g;       // index of the current g buffer (0..2)
  int nr_acc, nr_rej;
  int nr_ok;       // 1 if the Newton system of this iteration was solvable
  int max_iter;
  double tol;
  double l1_col;   // ||pi^T 1 - b||_1 at the last test
  double l1_row;
  double qsemi;    // Q_semi(f_k) of the last S4 pass
  double dq;       // Q_semi(f') - Q_semi(f_k) of the last trial
  double sum_wL;   // sum_j w_j L_j of the last pass
  double sum_wout; // sum_j w_j out_j of the last pass
  double dot_vd_a; // <V Delta, a>
  double sum_af;   // <f_k, a> after the last row pass
  int numeric;     // count of non-finite outputs seen
  int body_runs;   // executions of the current device loop body (hard-capped)
  int body_cap;
  // mode computation
  int eig_iter, eig_done, eig_max_iter, eig_fail;
  double eig_tol, eig_resid;
  int total_iters;
  int nr_degenerate;   // set when the SK-NR products saw exponentials out of range
  double stall_l1;     // L1 error at the last stall checkpoint of this level
  int stall_at;        // iteration of the next stall checkpoint
  long long trace_n;   // iteration records written to Prob::trace (all levels)
};

// Split arrays of one potential buffer (see eot_device.cuh).
struct Split {
  float* A;   // H(p + eps log w) + M     (reduction-side use)
  float* AL;  // L(p + eps log w)
  float* K;   // M - H(p)                 (output-side shift use)
  float* KL;  // L(p)
  // On-the-fly cost (EOT_PREC_SPLIT_TC): squared norms |pt|^2 of the side's
  // points; then K + KL = k2 (p - |pt|^2) split on the 2^-q grid (log2 units,
  // the same split for both sides, so that K_i + K_j is exact), A = the
  // side's weight (float) and AL = 0.
  const double* nrm;
};

// Everything the pass kernels need for one problem; lives in device memory.
struct Prob {
  int n, m;
  const float* C;          // n x m row-major
  const double *a, *b;     // weights
  const double *loga, *logb;
  double eps;
  float k2;                // log2(e) / eps, rounded to float32
  float k2lo;              // log2(e) / eps - k2.  The iteration's passes use k2 alone: they
                           // solve the problem at eps' = 1/(k2 ln 2), within 6e-8 relative
                           // of eps (a marginal error at eps of that relative size times a
                           // row's entropy).  The evaluation passes that verify a result
                           // add t k2lo, so the verification is at eps itself.
  float M;                 // magic constant 1.5 * 2^(23-q)
  double qscale, qinv;     // 2^q, 2^-q
  double* f[2];
  double* g[3];
  Split rs[2];
  Split cs[3];
  float* Lrow;             // natural-log marginal ratio of the last row pass (n)
  float* Lcol;             // ... of the last column pass (m)
  // column pass tiling
  int nstripe, rows_per_stripe, ncolblk;
  float2* part_col;        // [nstripe][m]
  unsigned* cnt_col;       // [ncolblk]
  double* acc_col;         // [ncolblk][4]
  // row pass tiling
  int nseg, cols_per_seg, nrowblk;
  float2* part_row;        // [nseg][n]
  unsigned* cnt_row;       // [nrowblk]
  double* acc_row;         // [nrowblk][4]
  unsigned* gcnt;          // [4] grid-level arrival counters
  // staged stream passes (stream.cu): grid sizes (0: not used), contributor
  // slots per output block, partial states, arrival counters, block sums
  CUtensorMap tmC;         // 2-D tensor map of C (box 128 columns x 32 rows), when used
  CUtensorMap tmCr;        // the same, box 32 columns x 128 rows, 128-byte swizzle
  int has_tmC;             // tmC encoded for this C
  int sk_gcol, sk_grow;
  int sk_slots_col, sk_slots_row;
  float2* sk_part_col;     // [ceil(m/128)][sk_slots_col][128]
  float2* sk_part_row;     // [ceil(n/32)][sk_slots_row][32]
  unsigned* sk_cnt_col;    // [ceil(m/128)]
  unsigned* sk_cnt_row;    // [ceil(n/32)]
  double* sk_acc_col;      // [ceil(m/32)][4] (per 128-column block, or per 32-column unit)
  double* sk_acc_row;      // [ceil(n/32)][4]
  unsigned* gbar;          // [2] grid barrier of the cooperative Sinkhorn loop
  unsigned long long wait_ns;   // bound of a grid-barrier wait (globaltimer ns)
  int stall_window;        // iterations between stall checkpoints (0: none)
  // on-the-fly cost (EOT_PREC_SPLIT_TC): C_ij = |x_i|^2 + |y_j|^2 - 2 x_i.y_j
  // with the Gram products on the tensor cores (3xTF32, float32 accumulation)
  int gram;                // 1 in that mode
  CUtensorMap tmXh, tmXl;  // TF32 high / low parts of X (n x 64, zero padded)
  CUtensorMap tmYh, tmYl;  // ... of Y (m x 64)
  const double* nX;        // |x_i|^2 (n)
  const double* nY;        // |y_j|^2 (m)
  int gm_grow, gm_gcol, gm_slots_row, gm_slots_col;
  float2* gm_part_row;     // [ceil(n/128)][gm_slots_row][128]
  float2* gm_part_col;     // [ceil(m/128)][gm_slots_col][128]
  unsigned* gm_cnt_row;    // [ceil(n/128)]
  unsigned* gm_cnt_col;    // [ceil(m/128)]
  double* gm_acc_row;      // [ceil(n/128)][4]
  double* gm_acc_col;      // [ceil(m/128)][4]
  State* st;
  // SK-NR
  int ell;                 // number of modes (0: none)
  const float* V;          // n x ell (row-major), a-orthonormal
  float* W;                // m x ell: W_j = pi(f_k,h)^T V  (row j)
  float* Wpart;            // [nstripe][m][ell] partial unnormalised sums
  double* delta;           // ell: Newton step
  double* GV;              // ell x ell: V^T D_a V
  double* Va;              // ell: V^T a
  double* WtW;             // ell x ell: sum_j W_j W_j^T / b_j
  double* grad;            // ell: gradient on V
  double pot_bound;        // |potential| limit of the exact exponent formation
  // float64 passes (EOT_PREC_FP64)
  const double* C64;       // n x m float64 cost
  double* fA64[2];         // f + eps log a for each f buffer
  double* gA64[3];         // g + eps log b for each g buffer
  double2* part64_col;     // [nstripe][m]
  double2* part64_row;     // [nseg][n]
  int ncolblk64, nrowblk64;
  unsigned long long cond; // graph conditional handle of the enclosing device loop
  // plain-mode outputs
  double* out_plain;       // standalone transform output
  double* logratio_plain;
  // iteration trace (eot_solve_traced): ring of trace_cap records, or NULL
  TraceRec* trace;
  int trace_cap;
};

// Arguments of the accumulating passes (accum.cu).
struct AccArgs {
  const Prob* P;
  int mode;              // 0: Op(pi)^T Z, 1: fused SK-NR column pass, 2: Op(pi) Z
  int k;                 // number of live columns of Z (<= kernel template width)
  const float* Z;        // (n or m) x k, row-major (Z for products, V for SK-NR)
  float* out;            // (m or n) x k output (products) or W (SK-NR)
  float* part;           // [nseg][len][K + 2] partial states
  unsigned* cnt;         // [nblk] arrival counters
  int nseg, seg_len, nblk;
  int fbuf, gbuf;        // which split buffers hold f and g (products)
  double* blkacc;        // [nblk][4]
  unsigned* gcnt;
  double* dw;            // (m) gradient weights d_j (SK-NR)
  double* wtw_part;      // [nblk][k*k + k] block partials (SK-NR)
  int cluster;           // staged kernel: merge a block's segments in a cluster (nseg <= 8)
  const int* skip;       // products: nonzero *skip makes the launch return at once (NULL: run)
};

// Debug build (-DEOT_DEBUG): a bounds check that fails records its site
// number (100 x unit + k) in its translation unit's debug word, the first
// failure winning, and the access it guards is skipped; the host reads every
// unit's word after a call (debug_site_<unit>, declared in api.cu) and fails
// the call with the site.  Without EOT_DEBUG a check is the constant true and
// the accessors return 0.
#ifdef EOT_DEBUG
#ifdef __CUDACC__
static __device__ unsigned g_eot_dbg_site;
__device__ __forceinline__ bool eot_check(bool ok, unsigned site) {
  if (!ok) atomicCAS(&g_eot_dbg_site, 0u, site);
  return ok;
}
#define EOT_CHECK(cond, site) ::eotk::eot_check((cond), (site))
#define EOT_DEBUG_UNIT(name)                                                   \
  unsigned debug_site_##name(bool reset) {                                     \
    unsigned v = 0;                                                            \
    if (cudaMemcpyFromSymbol(&v, g_eot_dbg_site, sizeof(v)) != cudaSuccess) {  \
      cudaGetLastError();                                                      \
      return 0u;                                                               \
    }                                                                          \
    if (reset && v) {                                                          \
      const unsigned z = 0;                                                    \
      cudaMemcpyToSymbol(g_eot_dbg_site, &z, sizeof(z));                       \
    }                                                                          \
    return v;                                                                  \
  }
#endif
#else
#define EOT_CHECK(cond, site) true
#define EOT_DEBUG_UNIT(name) \
  unsigned debug_site_##name(bool) { return 0u; }
#endif

#ifdef __CUDACC__
// Bytes of dynamic shared memory the running kernel was launched with.
__device__ __forceinline__ unsigned dyn_smem_bytes() {
  unsigned v;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}

// Iteration trace, written by the one thread that takes iteration `iter`'s
// stop decision: a new record (the oldest is overwritten once trace_cap are
// held); the Newton step of that iteration completes it (trace_trial).
__device__ inline void trace_test(const Prob& P, State* st, int iter, double l1, double qsemi) {
  if (!P.trace) return;
  TraceRec& r = P.trace[st->trace_n % P.trace_cap];
  r.eps = P.eps;
  r.l1 = l1;
  r.q_semi = qsemi;
  r.dq = __longlong_as_double(0x7ff8000000000000ll);   // NaN: no trial (yet)
  r.iter = iter;
  r.accepted = -1;
  st->trace_n += 1;
}
__device__ inline void trace_trial(const Prob& P, State* st, double dq, int accepted) {
  if (!P.trace || st->trace_n == 0) return;
  TraceRec& r = P.trace[(st->trace_n - 1) % P.trace_cap];
  r.dq = dq;
  r.accepted = accepted;
}

// Stop test of Algorithm 4.1 after iteration `iter` of a level with L1 marginal
// error l1 (one thread): 1 converged (l1 < tol), 2 iteration cap, 6 stalled,
// 0 go on.  Every `window` iterations l1 is compared with its value at the
// previous checkpoint; when it has not fallen below kStallRatio times that
// value the level stops: the error has reached the float32 passes' rounding
// floor, or falls so slowly (under 1% per window, over 200 windows per decade)
// that no practical iteration cap would reach the tolerance.  window 0 turns
// the check off.
constexpr double kStallRatio = 0.99;
__device__ inline int stop_code(State* st, double l1, int iter, double tol, int max_iter,
                                int window) {
  if (l1 < tol) return 1;
  if (iter >= max_iter) return 2;
  if (window > 0 && iter >= st->stall_at) {
    const bool stalled = !(l1 < kStallRatio * st->stall_l1);
    st->stall_l1 = l1;
    st->stall_at = iter + window;
    if (stalled) return 6;
  }
  return 0;
}
#endif

}  // namespace eotk
