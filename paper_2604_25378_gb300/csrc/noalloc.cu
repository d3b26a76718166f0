// Value and gradient of the sample oracle without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code that must not allocate in
// its steady state (a pre-sized memory budget, a hot loop inside a larger
// framework that owns the allocator) or code that hands this library only
// buffers it already owns.  mvsk_eval_noalloc serves them.  It runs the same
// fused value/gradient pass as mvsk_eval, with the pass's scratch (padded copy
// of x, per-CTA column and scalar partials, padded gradient, error word) in
// the fixed device array below instead of context memory.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "internal.h"
#include "mvsk.h"
#include "solver_kernels.cuh"

namespace {

// 8 MiB of scratch, resident on every GPU that loads the library until exit.
constexpr size_t kNoAllocDoubles = (size_t)1 << 20;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

mvsk_status noalloc_fail(mvsk_status st, const char* msg) {
  mvsk::set_last_error(msg);
  return st;
}

__global__ void k_pad_copy(const double* src, double* dst, int n, int ld) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ld; i += gridDim.x * blockDim.x)
    dst[i] = i < n ? src[i] : 0.0;
}

// f = -c1 mu^T x + T^-1 sum_b spart[b] (the value of Eq. operator-f).
__global__ void __launch_bounds__(mvsk::kVT) k_noalloc_value(const double* mu, const double* x, int n,
                                                             const double* spart, int G, double c1, double invT,
                                                             double* f) {
  __shared__ double scr[80];
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx += mu[i] * x[i];
  mx = mvsk::block_sum2(mx, 0.0, scr).x;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += spart[b];
    *f = -c1 * mx + s * invT;
  }
}

}  // namespace

extern "C" mvsk_status mvsk_eval_noalloc(const double* A, const double* mu, int64_t T, int64_t n, int64_t ld,
                                         const double c[4], const double* x, double* z, double* g, double* f,
                                         void* stream) {
  using namespace mvsk;
  if (A == nullptr || mu == nullptr || c == nullptr || x == nullptr || z == nullptr || g == nullptr ||
      f == nullptr)
    return noalloc_fail(MVSK_EINVAL, "mvsk_eval_noalloc: null argument");
  if (T < 1 || n < 1 || n > kMaxCols || ld < n || ld > kMaxCols || (ld % 2) != 0 ||
      (reinterpret_cast<uintptr_t>(A) % 16) != 0)
    return noalloc_fail(MVSK_EINVAL,
                        "mvsk_eval_noalloc: need T >= 1, 1 <= n <= ld <= 6144, ld even, A 16-byte aligned");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: no usable current device");
  cudaStream_t st = (cudaStream_t)stream;
  double* base = nullptr;
  {
    // One-time set-up per device, with that device current: the host-side
    // symbol is not a device address, so fetch the real one.
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: cudaGetSymbolAddress of the scratch array failed");
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    base = g_scratch_ptr[dev];
  }
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: device query failed");
  // Scratch layout (doubles): x padded [ld] | g padded [ld] | error word [8] | scalar partials [grid] | column partials [grid*ld].
  const size_t fixed = 2 * (size_t)ld + 8;
  if (fixed + (size_t)ld + 1 > kNoAllocDoubles)
    return noalloc_fail(MVSK_EINVAL, "mvsk_eval_noalloc: ld too large for the 8 MiB scratch array");
  long long grid = T < nsm ? T : nsm;
  const long long cap = (long long)((kNoAllocDoubles - fixed) / ((size_t)ld + 1));
  if (grid > cap) grid = cap;
  const long long rows_per_cta = (T + grid - 1) / grid;
  grid = (T + rows_per_cta - 1) / rows_per_cta;
  double* xpad = base;
  double* gpad = base + ld;
  int* err = reinterpret_cast<int*>(base + 2 * (size_t)ld);
  double* spart = base + fixed;
  double* part = spart + grid;
  if (rowpass_init_f64() != cudaSuccess)
    return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: kernel attribute set-up failed");
  int stages = 0;
  const size_t smem = rowpass_smem(P64, M_VALGRAD, 1, (int)ld, &stages);
  if (smem == 0) return noalloc_fail(MVSK_EINVAL, "mvsk_eval_noalloc: row too long for the pass");
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
    return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: clearing the error word failed");
  k_pad_copy<<<(int)((ld + 255) / 256), 256, 0, st>>>(x, xpad, (int)n, (int)ld);
  PassArgs a;
  memset(&a, 0, sizeof(a));
  a.A = A;
  a.T = T;
  a.ld = (int)ld;
  a.in[0] = xpad;
  a.rowout = z;
  a.c2 = c[1];
  a.c3 = c[2];
  a.c4 = c[3];
  a.rscale = 1.0;
  a.part = part;
  a.spart = spart;
  a.rows_per_cta = (int)rows_per_cta;
  a.stages = stages;
  a.err = err;
  if (rowpass_launch(P64, M_VALGRAD, 1, a, (int)grid, smem, st) != cudaSuccess)
    return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: pass launch failed");
  dim3 rg((unsigned)((ld + 255) / 256), 1);
  k_reduce_cols<double><<<rg, 256, 0, st>>>(part, (int)grid, 1, (int)ld, (int)n, 1.0 / (double)T, mu, -c[0], gpad,
                                            (size_t)ld, nullptr, nullptr);
  k_noalloc_value<<<1, kVT, 0, st>>>(mu, xpad, (int)n, spart, (int)grid, c[0], 1.0 / (double)T, f);
  if (cudaGetLastError() != cudaSuccess) return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: launch failed");
  if (cudaMemcpyAsync(g, gpad, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: copy of the gradient failed");
  if (cudaStreamSynchronize(st) != cudaSuccess)
    return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: stream synchronisation failed");
  int e = 0;
  if (cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: reading the error word failed");
  if (e != 0) return noalloc_fail(MVSK_ECUDA, "mvsk_eval_noalloc: an in-kernel bounded wait ran out");
  return MVSK_OK;
}
