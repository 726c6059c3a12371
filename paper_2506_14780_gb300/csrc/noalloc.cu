// eot_ctransform_noalloc: the (C, eps)-transform of eot_ctransform for callers
// that may not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a fixed device
// memory pool owned by another allocator (a framework's caching allocator or
// an embedding application that sized the whole device at start-up), where a
// foreign allocation can fail or break the pool's budget; and latency-critical
// loops, where cudaMalloc / cudaFree may synchronise the device.  This entry
// point keeps all of its temporaries (problem descriptor, split arrays,
// per-segment partial sums, arrival counters) in one file-scope device array,
// g_noalloc_scratch, of kNoAllocScratchBytes (4 MiB), which every GPU that
// loads the library holds until the process exits.  It launches the same pass
// kernels as eot_ctransform, on the caller's stream, and never allocates: no
// cudaMalloc, cudaFree, cudaMallocHost, stream or event creation.
//
// Limits: n, m <= kNoAllocMaxDim (16384) and the tiling's partial sums must
// fit the array; larger sizes return EOT_EINVAL before any device work.
// The first call on a device looks up the array's device address
// (cudaGetSymbolAddress) with that device current; make that first call before
// any stream capture.  Every call synchronises the caller's stream before it
// returns (it reads the cost's range back to the host to place the exponent
// grid), also when it fails after enqueueing work.  All calls share the one
// array and it keeps the last call's contents: calls that overlap on the GPU
// (on different streams or threads without ordering) race and corrupt each
// other.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "eot.h"
#include "eot_internal.h"

namespace eotk {

cudaError_t launch_col_pass(const Prob* dP, const Prob& hP, int mode, cudaStream_t s);
cudaError_t launch_row_pass(const Prob* dP, const Prob& hP, int mode, cudaStream_t s);
cudaError_t launch_split(const Prob* dP, const double* p, const double* logw, int len, Split so,
                         cudaStream_t s);
__global__ void cost_stats_kernel(size_t, const float*, unsigned*, unsigned*);
__global__ void cost_stats_f64_kernel(size_t, const double*, unsigned long long*, unsigned*);
__global__ void weights_kernel(int, const double*, double*, double*, unsigned*, int);

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;
constexpr int kNoAllocMaxDim = 16384;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[128] = {nullptr};

// the thread-local message behind eot_last_error (api.cu)
void set_last_error(const std::string& msg);

static eot_status na_fail(eot_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

// Sub-allocation inside the static array (offsets only; nothing is allocated).
struct Carve {
  char* base;
  size_t off = 0;
  size_t cap;
  bool ok = true;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += std::max<size_t>(count, 1) * sizeof(T);
    if (off > cap) ok = false;
    return p;
  }
};

}  // namespace eotk

using namespace eotk;

extern "C" eot_status eot_ctransform_noalloc(eot_side side, int32_t n, int32_t m, const float* C,
                                             const double* pot, const double* w,
                                             const double* shift, double eps, double* out,
                                             double* log_ratio, void* stream) {
  if (!C || !pot || !w || !out) return na_fail(EOT_EINVAL, "C, pot, w and out are required");
  if (!(eps > 0.0) || !std::isfinite(eps)) return na_fail(EOT_EINVAL, "eps must be finite and > 0");
  if (side != EOT_SIDE_COL && side != EOT_SIDE_ROW) return na_fail(EOT_EINVAL, "bad side");
  if (n < 1 || m < 1) return na_fail(EOT_EINVAL, "n and m must be >= 1");
  if (n > kNoAllocMaxDim || m > kNoAllocMaxDim)
    return na_fail(EOT_EINVAL, "eot_ctransform_noalloc: n and m must be <= 16384 (static scratch)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128)
    return na_fail(EOT_ECUDA, "no usable CUDA device");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return na_fail(EOT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_noalloc_ptr[dev] = p;
    }
    base = g_noalloc_ptr[dev];
  }
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return na_fail(EOT_ECUDA, "cudaDeviceGetAttribute failed");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto cdiv = [](long long a, long long b) { return (int)((a + b - 1) / b); };

  // tiling of the two pass kernels (same rules as the solver)
  Prob P{};
  P.n = n;
  P.m = m;
  const int target = 4 * nsm;
  P.ncolblk = cdiv(m, kColTile);
  P.nstripe = std::max(1, std::min(cdiv(n, 32), (target + P.ncolblk - 1) / P.ncolblk));
  P.rows_per_stripe = cdiv(cdiv(n, P.nstripe), 8) * 8;
  P.nstripe = cdiv(n, P.rows_per_stripe);
  P.nrowblk = cdiv(n, kRowTile);
  P.nseg = std::max(1, std::min(cdiv(m, 128), (target + P.nrowblk - 1) / P.nrowblk));
  P.cols_per_seg = cdiv(cdiv(m, P.nseg), 128) * 128;
  P.nseg = cdiv(m, P.cols_per_seg);

  Carve cv{reinterpret_cast<char*>(base), 0, kNoAllocScratchBytes};
  Prob* dP = cv.take<Prob>(1);
  State* dSt = cv.take<State>(1);
  unsigned* stats = cv.take<unsigned>(4);
  unsigned long long* pmax = cv.take<unsigned long long>(1);
  double* wa = cv.take<double>(n);
  double* wb = cv.take<double>(m);
  P.a = cv.take<double>(n);
  P.loga = cv.take<double>(n);
  P.b = cv.take<double>(m);
  P.logb = cv.take<double>(m);
  for (int k = 0; k < 2; ++k) {
    P.f[k] = cv.take<double>(n);
    P.g[k] = cv.take<double>(m);
  }
  P.rs[0] = Split{cv.take<float>(n), cv.take<float>(n), cv.take<float>(n), cv.take<float>(n)};
  P.cs[0] = Split{cv.take<float>(m), cv.take<float>(m), cv.take<float>(m), cv.take<float>(m)};
  P.Lrow = cv.take<float>(n);
  P.Lcol = cv.take<float>(m);
  P.part_col = cv.take<float2>((size_t)P.nstripe * m);
  P.cnt_col = cv.take<unsigned>(P.ncolblk);
  P.acc_col = cv.take<double>((size_t)P.ncolblk * 4);
  P.part_row = cv.take<float2>((size_t)P.nseg * n);
  P.cnt_row = cv.take<unsigned>(P.nrowblk);
  P.acc_row = cv.take<double>((size_t)P.nrowblk * 4);
  P.gcnt = cv.take<unsigned>(4);
  if (!cv.ok)
    return na_fail(EOT_EINVAL, "eot_ctransform_noalloc: problem too large for the static scratch");
  P.st = dSt;

  // On a failure after work was enqueued, wait for that work before
  // returning: a retry (on any stream) must not overlap kernels that still
  // use the shared array.  The wait's own status is not needed.
#define NA_TRY(expr)                                                                  \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) {                                                          \
      (void)cudaStreamSynchronize(s);                                                 \
      return na_fail(EOT_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));  \
    }                                                                                 \
  } while (0)

  // everything that must start at zero: state, counters, the unused weights
  NA_TRY(cudaMemsetAsync(dSt, 0, sizeof(State), s));
  NA_TRY(cudaMemsetAsync(stats, 0, 4 * sizeof(unsigned), s));
  NA_TRY(cudaMemsetAsync(pmax, 0, sizeof(unsigned long long), s));
  NA_TRY(cudaMemsetAsync(P.cnt_col, 0, P.ncolblk * sizeof(unsigned), s));
  NA_TRY(cudaMemsetAsync(P.cnt_row, 0, P.nrowblk * sizeof(unsigned), s));
  NA_TRY(cudaMemsetAsync(P.gcnt, 0, 4 * sizeof(unsigned), s));
  const bool col = side == EOT_SIDE_COL;
  const int nred = col ? n : m, nout = col ? m : n;
  // weights of the reduction side (as given, not renormalised); zeros elsewhere
  if (col) {
    NA_TRY(cudaMemcpyAsync(wa, w, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    weights_kernel<<<1, 256, 0, s>>>(n, wa, const_cast<double*>(P.a), const_cast<double*>(P.loga),
                                     stats + 2, 0);
    NA_TRY(cudaMemsetAsync(const_cast<double*>(P.b), 0, m * sizeof(double), s));
    NA_TRY(cudaMemsetAsync(const_cast<double*>(P.logb), 0, m * sizeof(double), s));
  } else {
    NA_TRY(cudaMemcpyAsync(wb, w, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    weights_kernel<<<1, 256, 0, s>>>(m, wb, const_cast<double*>(P.b), const_cast<double*>(P.logb),
                                     stats + 2, 0);
    NA_TRY(cudaMemsetAsync(const_cast<double*>(P.a), 0, n * sizeof(double), s));
    NA_TRY(cudaMemsetAsync(const_cast<double*>(P.loga), 0, n * sizeof(double), s));
  }
  // exponent grid from max |C| and the potentials' range (host read-back into
  // stack variables: a synchronous copy, no pinned buffer)
  const size_t nm = (size_t)n * m;
  const int gb = (int)std::min<long long>(((long long)nm + 255) / 256, 8LL * nsm);
  cost_stats_kernel<<<gb, 256, 0, s>>>(nm, C, stats, stats + 1);
  cost_stats_f64_kernel<<<cdiv(nred, 256), 256, 0, s>>>(nred, pot, pmax, stats + 3);
  if (shift) cost_stats_f64_kernel<<<cdiv(nout, 256), 256, 0, s>>>(nout, shift, pmax, stats + 3);
  NA_TRY(cudaGetLastError());
  unsigned hs[4];
  unsigned long long hpm = 0;
  NA_TRY(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, s));
  NA_TRY(cudaMemcpyAsync(&hpm, pmax, sizeof(hpm), cudaMemcpyDeviceToHost, s));
  NA_TRY(cudaStreamSynchronize(s));
  if (hs[2]) return na_fail(EOT_EINVAL, "weights must be positive and finite");
  if (hs[1]) return na_fail(EOT_EINVAL, "cost has non-finite entries");
  if (hs[3]) return na_fail(EOT_EINVAL, "potentials have non-finite entries");
  float cm;
  std::memcpy(&cm, &hs[0], 4);
  double pm;
  std::memcpy(&pm, &hpm, 8);
  const double R = 4.0 * ((double)cm + pm + 40.0 * eps) + 1e-30;
  int q = 22 - (int)std::ceil(std::log2(R));
  q = std::max(-100, std::min(q, 60));
  P.C = C;
  P.qscale = std::ldexp(1.0, q);
  P.qinv = std::ldexp(1.0, -q);
  P.M = (float)(1.5 * std::ldexp(1.0, 23 - q));
  P.pot_bound = std::ldexp(1.0, 22 - q) / 2.0 - cm;
  P.eps = eps;
  P.k2 = (float)(1.0 / (eps * std::log(2.0)));
  P.k2lo = (float)(1.0 / (eps * std::log(2.0)) - (double)P.k2);
  double* redbuf = col ? P.f[0] : P.g[0];
  double* outbuf = col ? P.g[0] : P.f[0];
  NA_TRY(cudaMemcpyAsync(redbuf, pot, nred * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (shift) NA_TRY(cudaMemcpyAsync(outbuf, shift, nout * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else NA_TRY(cudaMemsetAsync(outbuf, 0, nout * sizeof(double), s));
  const int passes = shift ? 1 : 2;
  for (int pass = 0; pass < passes; ++pass) {
    const bool final_pass = pass == passes - 1;
    P.out_plain = final_pass ? out : (col ? P.g[1] : P.f[1]);
    P.logratio_plain = final_pass ? log_ratio : nullptr;
    // the descriptor is read by the kernels from device memory (pageable copy)
    NA_TRY(cudaMemcpyAsync(dP, &P, sizeof(Prob), cudaMemcpyHostToDevice, s));
    NA_TRY(launch_split(dP, P.f[0], P.loga, n, P.rs[0], s));
    NA_TRY(launch_split(dP, P.g[0], P.logb, m, P.cs[0], s));
    NA_TRY(col ? launch_col_pass(dP, P, MODE_PLAIN, s) : launch_row_pass(dP, P, MODE_PLAIN, s));
    if (!final_pass)
      NA_TRY(cudaMemcpyAsync(outbuf, col ? P.g[1] : P.f[1], nout * sizeof(double),
                             cudaMemcpyDeviceToDevice, s));
    // the host descriptor is overwritten by the next pass: wait for this copy
    NA_TRY(cudaStreamSynchronize(s));
  }
#undef NA_TRY
  return EOT_OK;
}
