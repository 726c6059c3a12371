// Internal layout of the persistent batched Sinkhorn (batch.cu), shared with
// the host code that fills it (api.cu).
#pragma once
#include <stddef.h>
#include "eot_internal.h"

namespace eotk {

constexpr int kBThreads = 256;
constexpr int kBMaxLev = 64;
constexpr int kBMaxGang = 32;
constexpr int kBRowU = 8;                 // 4-column groups a lane loads per step (row pass)
constexpr double kBCostPerCta = 1.25 * 1024 * 1024;   // floor of the gang sizes: cost bytes per CTA
constexpr unsigned long long kWaitNsDefault = 30000000000ull;   // 30 s bound of a device wait

struct BatchOut {
  int status;        // 1 converged, 2 iteration cap, 3 numeric, 4 gang wait gave up,
                     // 6 the last level's L1 error stalled
  int iters, total_iters, levels, verify_rounds, pad;
  double row_l1, col_l1, q_dual, q_semi, dual_gap, gauge;
  unsigned long long t_begin, t_end, t_last_level;
};

// Tiles of the batch passes (BatchTask::tile, picked per size class of m by
// the host's tuner): bit 0, two columns a lane in the column half-step
// (64-column blocks) instead of four (128); bit 1, at least eight rows a warp
// per chunk of the row half-step instead of four.  No tile changes a result.
constexpr int kBTiles = 4;

struct BatchTask {
  int n, m, pitch, nlev, G, max_iter;
  int tile;                       // pass tiles (kBTiles variants)
  int lpr;                        // lanes per row of the row pass (batch_lpr(m))
  const float* C;                 // n x pitch
  const double *a, *b, *loga, *logb;
  const float *af, *bf;           // the weights in float32 (L1 sums)
  double* f;                      // n
  double* g[2];                   // m, double-buffered
  Split fs;                       // split arrays of f
  Split gsp[2];                   // of g[0], g[1]
  float *Lrow, *Lcol;
  double *f_out, *g_out;
  unsigned* bar;                  // [2]: arrivals, generation
  unsigned long long wait_ns;     // bound of a gang-barrier wait (globaltimer ns)
  int stall_window;               // iterations between stall checkpoints (0: none)
  unsigned* flag;                 // numeric flag of the problem (0 / 1)
  BatchOut* out;
  double tol_level, tol_last, tol_verify;
  double qscale, qinv, pot_bound;
  float M;
  double eps[kBMaxLev];
};

struct BatchIn {
  int n, m, d, pitch, normalize, givenC;
  int trans;                   // given cost read transposed (Cin is m x n)
  const float *X, *Y;          // points (d > 0)
  const float* Cin;            // given cost, n x m (d == 0)
  const double *win_a, *win_b; // weights as given
  double *a, *b, *loga, *logb; // normalised weights and their logs
  float *af, *bf;              // the normalised weights in float32
  float* C;                    // n x pitch
  unsigned long long* cmax;    // float64 bits of max C (or max |C|)
  unsigned* bad;               // [0] weights, [1] cost
};


// Lanes that reduce one row in the row pass: the smallest power of two (at
// most 32) for which a lane holds at most kBRowU of the row's 4-column groups
// per step.  A function of m alone: every row sums in the same order whatever
// the gang.
inline __host__ __device__ int batch_lpr(int m) {
  const int ng = (m + 3) >> 2;
  int L = 1;
  while (L < 32 && L * kBRowU < ng) L *= 2;
  return L;
}

int batch_ctas_per_sm();
cudaError_t launch_batch_setup(const BatchIn* d_in, int count, int maxrows, cudaStream_t s);
cudaError_t launch_batch_sk(const BatchTask* d_tasks, const int2* d_slots, int nslots,
                            unsigned* d_next, int grid, cudaStream_t s);

}  // namespace eotk
