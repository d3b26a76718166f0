// Shared device helpers: bulk-TMA staging with mbarriers (bounded waits),
// block reductions, psi derivatives.  sm_103a only.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mvsk {

constexpr int kThreads = 512;           // threads per row-pass CTA
constexpr int kWarps = kThreads / 32;
constexpr int kMaxCols = 6144;          // largest n supported by the streaming passes
constexpr int kPad = 64;                // leading dimension of A is n rounded up to 64 elements
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on any in-kernel wait

// Error bits written by kernels into the context's error word.
enum : int { kErrWaitTimeout = 1, kErrDrainTimeout = 2, kErrNonFinite = 4 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// One contiguous global -> shared bulk copy completing on `bar` (16-byte
// aligned addresses, size a multiple of 16 bytes).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar`, giving up after kWaitNs.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum over blockDim.x threads (multiple of 32) in a fixed order.
// `scratch` holds >= 33 doubles (slot 32 broadcasts the total).  All threads
// receive the result.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < nw ? scratch[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) scratch[32] = t;
  }
  __syncthreads();
  return scratch[32];
}

// Reductions of the single-CTA-per-instance kernels (up to 1024 threads).
// The values are staged in shared memory; the nw = blockDim.x / 32 rows are
// folded column by column (lane l takes entries l, l + 32, ...) and finished
// with one 5-level shuffle: about nw + 5 warp-wide FP64 operations per value
// instead of a shuffle tree in every warp (5 per warp, ~160 for 1024 threads)
// on a pipe of ~2 FMA/clk/SM.  A warp-wide FP64 instruction occupies its
// scheduler's FP64 pipe ~64 cycles, so the sums (block_sum2_fin,
// block_sum2c_fin) fold in two stages: warps 0..3, one per scheduler, each a
// quarter of the rows, then warp 0 the four partial rows.  Staging: 2 x 1024
// doubles and 1024 ints per kernel that uses them, plus the second stage.
__device__ __forceinline__ double* red_stage() {
  __shared__ double st[2 * 1024];
  return st;
}
__device__ __forceinline__ int* red_stage_i() {
  __shared__ int sti[1024];
  return sti;
}
// Second stage of the folds below: warps 0..3 (one per scheduler) each fold a
// quarter of the staged rows, so that the FP64 additions of the first stage
// run on four pipes at once; 2 x 128 doubles and 128 ints.
__device__ __forceinline__ double* red_stage2() {
  __shared__ double st2[256];
  return st2;
}
__device__ __forceinline__ int* red_stage2_i() {
  __shared__ int st2i[128];
  return st2i;
}

__device__ __forceinline__ double block_min(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* st = red_stage();
  __syncthreads();
  st[threadIdx.x] = v;
  __syncthreads();
  if (warp == 0) {
    double t = INFINITY;
    for (int k = 0; k < nw; ++k) t = fmin(t, st[k * 32 + lane]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (lane == 0) scratch[32] = t;
  }
  __syncthreads();
  return scratch[32];
}

// Block-wide arg-max (value, index); ties take the smallest index.
__device__ __forceinline__ void block_argmax(double& v, int& idx, double* sv, int* si) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* st = red_stage();
  int* sti = red_stage_i();
  __syncthreads();
  st[threadIdx.x] = v;
  sti[threadIdx.x] = idx;
  __syncthreads();
  if (warp == 0) {
    double t = -INFINITY;
    int ti = 0x7fffffff;
    for (int k = 0; k < nw; ++k) {
      const double ov = st[k * 32 + lane];
      const int oi = sti[k * 32 + lane];
      if (ov > t || (ov == t && oi < ti)) {
        t = ov;
        ti = oi;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, t, o);
      const int oi = __shfl_xor_sync(0xffffffffu, ti, o);
      if (ov > t || (ov == t && oi < ti)) {
        t = ov;
        ti = oi;
      }
    }
    if (lane == 0) {
      sv[32] = t;
      si[32] = ti;
    }
  }
  __syncthreads();
  v = sv[32];
  idx = si[32];
}

// psi and its derivatives (Prop. 2, Eqs. operator-grad/hvp/third).
struct Psi {
  double c2, c3, c4;
  __device__ __forceinline__ double f(double s) const { return s * s * (c2 - s * (c3 - c4 * s)); }
  __device__ __forceinline__ double d1(double s) const { return s * (2.0 * c2 - s * (3.0 * c3 - 4.0 * c4 * s)); }
  __device__ __forceinline__ double d2(double s) const { return 2.0 * c2 - s * (6.0 * c3 - 12.0 * c4 * s); }
  __device__ __forceinline__ double d3(double s) const { return -6.0 * c3 + 24.0 * c4 * s; }
};

// Shape of one tensor-core product restricted to the union U of the working
// faces of a lockstep batch (its runtime extents depend on |U|).
struct UProd {
  int rows_dyn;  // 1: output rows = |U| (A^T products), 0: rows fixed = M
  int M;         // fixed rows (rows_dyn = 0)
  int K;         // fixed K (rows_dyn = 1), else K = |U| rounded up to 64
  int mrows;     // rows per CTA tile
  int nt;        // N tiles
  int slots;     // resident CTAs of the machine
  int tensor;    // tensor-bound (split-K by the time model) or bandwidth-bound
  int smax;      // largest split count the grid and the partial buffer allow
};

}  // namespace mvsk
