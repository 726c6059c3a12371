// Internal layout of the persistent batched Sinkhorn (batch.cu), shared with
// the host code that fills it (api.cu).
#pragma once
#include <stddef.h>
#include "eot_internal.h"

namespace eotk {

constexpr int kBThreads = 256;
constexpr int kBMaxLev = 64;
constexpr int kBPart = 16;                // partial sums per rank: [0..3] column pass,
                                          // [8..11] row evaluation, [12..15] scores
constexpr int kBMaxGang = 32;
constexpr unsigned long long kBWaitNs = 30000000000ull;   // 30 s bound of a gang wait

struct BatchOut {
  int status;        // 1 converged, 2 iteration cap, 3 numeric, 4 gang wait gave up
  int iters, total_iters, levels, verify_rounds, pad;
  double row_l1, col_l1, q_dual, q_semi, dual_gap, gauge;
  unsigned long long t_begin, t_end, t_last_level;
};

struct BatchTask {
  int n, m, pitch, nlev, G, max_iter;
  const float* C;                 // n x pitch
  const double *a, *b, *loga, *logb;
  double* f;                      // n
  double* g[2];                   // m, double-buffered
  Split fs;                       // split arrays of f
  Split gsp[2];                   // of g[0], g[1]
  float *Lrow, *Lcol;
  double *f_out, *g_out;
  unsigned* bar;                  // [2]: arrivals, generation
  double* part;                   // [G][kBPart]
  BatchOut* out;
  double tol_level, tol_last, tol_verify;
  double qscale, qinv, pot_bound;
  float M;
  double eps[kBMaxLev];
};

struct BatchIn {
  int n, m, d, pitch, normalize, givenC;
  const float *X, *Y;          // points (d > 0)
  const float* Cin;            // given cost, n x m (d == 0)
  const double *win_a, *win_b; // weights as given
  double *a, *b, *loga, *logb; // normalised weights and their logs
  float* C;                    // n x pitch
  unsigned long long* cmax;    // float64 bits of max C (or max |C|)
  unsigned* bad;               // [0] weights, [1] cost
};


int batch_ctas_per_sm();
cudaError_t launch_batch_setup(const BatchIn* d_in, int count, int maxrows, cudaStream_t s);
cudaError_t launch_batch_sk(const BatchTask* d_tasks, const int2* d_slots, int nslots,
                            unsigned* d_next, int grid, cudaStream_t s);

}  // namespace eotk
