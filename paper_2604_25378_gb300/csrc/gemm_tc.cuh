// BF16 x BF16 -> FP32 tensor-core GEMM for sm_103a (tcgen05 + TMA + TMEM).
//
//   C[m, n] = sum_k A[m, k] B[n, k]      (A: M x K, B: N x K, both K-major BF16)
//
// One 128 x BN output tile per CTA of 128 threads:
//   * warp 0 lane 0 streams 128x64 (A) and BNx64 (B) BF16 tiles with TMA
//     (128-byte swizzle) into a 4-stage shared-memory ring (mbarrier full/empty);
//   * warp 1 lane 0 issues tcgen05.mma (kind::f16, M=128, N=BN, K=16 per
//     instruction) into a TMEM accumulator of BN FP32 columns and commits each
//     stage back to the producer;
//   * all four warps read the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31 = output rows) and hand 32-column slices to the epilogue.
// Every wait is bounded (kWaitNs); a wait that runs out sets the error word,
// the CTA drains its in-flight copies, frees its TMEM and returns.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace mvsk {

constexpr int kTcBM = 128, kTcBK = 64, kTcStages = 4;

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile of 128-byte rows written by
// TMA with 128-byte swizzle (8-row atoms of 1024 bytes, atoms 1024 bytes apart).
__device__ __forceinline__ uint64_t umma_desc_sw128(const void* tile) {
  const uint32_t a = smem_u32(tile);
  uint64_t d = 0;
  d |= (uint64_t)((a >> 4) & 0x3FFFu);        // start address (16-byte units)
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 1024 bytes between 8-row atoms
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int CW>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[CW]) {
  if constexpr (CW == 32) tmem_ld32(taddr, v);
  else tmem_ld16(taddr, v);
}

template <int BN, int STAGES = kTcStages, int MT = 1>
__host__ __device__ constexpr size_t tc_smem_bytes() {
  return 1024 /* alignment slack */ + (size_t)STAGES * (MT * kTcBM * kTcBK * 2 + BN * kTcBK * 2) + 256;
}

// Epilogue: FP64 store C[m*ldc + n] = alpha * acc for m < M, n < N.
struct EpiStoreF64 {
  double* C;
  long long ldc;
  double alpha;
  int M, N;
  template <int CW>
  __device__ __forceinline__ void operator()(int m, int n0, const float (&v)[CW], int) const {
    if (m >= M) return;
    double* row = C + (size_t)m * ldc;
#pragma unroll
    for (int i = 0; i < CW; ++i)
      if (n0 + i < N) row[n0 + i] = alpha * (double)v[i];
  }
};

// Epilogue of split-K products: FP32 partial part[(kz*N + n)*ldp + m] = acc
// (m < M, n < N); lanes hold consecutive m, so each column store is coalesced.
struct EpiPartT {
  float* part;
  long long ldp;
  int M, N;
  template <int CW>
  __device__ __forceinline__ void operator()(int m, int n0, const float (&v)[CW], int kz) const {
    if (m >= M) return;
#pragma unroll
    for (int i = 0; i < CW; ++i)
      if (n0 + i < N) part[((size_t)kz * N + n0 + i) * ldp + m] = v[i];
  }
};

// Epilogue of the first product of a batched Hessian-vector block (no
// split-K): S^T[q][t] = bf16(h_{q / nc}[t] * acc) for the columns q < N of the
// N x T output, h in FP32 (T-strided per instance).
struct EpiHvp1 {
  __nv_bfloat16* S;
  long long Tp;
  const float* Hf;
  int T, N, nc;
  template <int CW>
  __device__ __forceinline__ void operator()(int m, int n0, const float (&v)[CW], int) const {
    if (m >= T) return;
    __nv_bfloat16* __restrict__ out = S;
    const float* __restrict__ h = Hf;
    // all h loads of the chunk first (independent, read-only path), then the stores
    float hv[CW];
    int b = n0 / nc, j = n0 - b * nc;
#pragma unroll
    for (int i = 0; i < CW; ++i) {
      hv[i] = n0 + i < N ? __ldg(h + (size_t)b * T + m) : 0.f;
      if (++j == nc) {
        j = 0;
        ++b;
      }
    }
#pragma unroll
    for (int i = 0; i < CW; ++i)
      if (n0 + i < N) out[(size_t)(n0 + i) * Tp + m] = __float2bfloat16(hv[i] * v[i]);
  }
};

// Split-K: CTA (x, y, z) computes output tile (n0 = x*BN, m0 = y*128*MT) over the
// k-tiles [z*ktps, min(nk, (z+1)*ktps)) and hands the epilogue its z.  MT = 2
// stacks two 128-row subtiles that share each B tile (accumulators at TMEM
// columns 0 and BN): a third fewer operand bytes per MAC than MT = 1.
template <int BN, int STAGES, class Epi, int MT = 1>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                                                    int ktps, Epi epi, int* err, const int* skip,
                                                    const int* live) {
  static_assert(BN == 16 || BN == 32 || BN == 64 || BN == 128 || BN == 192 || BN == 256, "unsupported N tile");
  static_assert(MT == 1 || (MT == 2 && BN >= 32), "two subtiles need BN >= 32");
  constexpr int kTcStages = STAGES;
  constexpr uint32_t TUSED = MT * (BN < 32 ? 32 : BN);
  constexpr uint32_t TCOLS = TUSED <= 32 ? 32 : TUSED <= 64 ? 64 : TUSED <= 128 ? 128 : TUSED <= 256 ? 256 : 512;
  constexpr int CW = BN < 32 ? BN : 32;
  if (skip != nullptr && *skip != 0) return;
  if (live != nullptr && *live == 0) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int ABYTES = MT * kTcBM * kTcBK * 2;
  constexpr int BBYTES = BN * kTcBK * 2;
  unsigned char* sA = sm;
  unsigned char* sB = sm + (size_t)kTcStages * ABYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + (size_t)kTcStages * BBYTES);
  uint64_t* empty = full + kTcStages;
  uint64_t* done = empty + kTcStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int s_abort;
  __shared__ int s_issued;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcBM * MT, n0 = blockIdx.x * BN;
  const int nk_all = (K + kTcBK - 1) / kTcBK;
  const int kt0 = blockIdx.z * ktps;
  const int kt1 = kt0 + ktps < nk_all ? kt0 + ktps : nk_all;
  const int nk = kt1 > kt0 ? kt1 - kt0 : 0;
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_issued = 0;
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nk; ++i) {
      const int s = i % kTcStages;
      if (i >= kTcStages && !mbar_wait_bounded(&empty[s], (uint32_t)(((i / kTcStages) - 1) & 1))) {
        s_abort = 1;
        atomicOr(err, kErrWaitTimeout);
        break;
      }
      if (s_abort) break;
      mbar_expect_tx(&full[s], ABYTES + BBYTES);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
        tma_load_2d(sA + (size_t)s * ABYTES + (size_t)mt * kTcBM * kTcBK * 2, &tmA, (kt0 + i) * kTcBK,
                    m0 + mt * kTcBM, &full[s]);
      tma_load_2d(sB + (size_t)s * BBYTES, &tmB, (kt0 + i) * kTcBK, n0, &full[s]);
      s_issued = i + 1;
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16_f32(kTcBM, BN);
    for (int i = 0; i < nk; ++i) {
      const int s = i % kTcStages;
      if (!mbar_wait_bounded(&full[s], (uint32_t)((i / kTcStages) & 1))) {
        s_abort = 1;
        atomicOr(err, kErrWaitTimeout);
        break;
      }
      tc_fence_after();
      const uint64_t db = umma_desc_sw128(sB + (size_t)s * BBYTES);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const uint64_t da = umma_desc_sw128(sA + (size_t)s * ABYTES + (size_t)mt * kTcBM * kTcBK * 2);
          umma_bf16(tmem + (uint32_t)(mt * (BN < 32 ? 32 : BN)), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk),
                    idesc, (i > 0 || kk > 0) ? 1u : 0u);
        }
      umma_commit(&empty[s]);
    }
    umma_commit(done);  // arrives once every MMA issued above has completed
  }
  __syncwarp();
  // Epilogue: accumulator rows = TMEM lanes.
  const bool ok = mbar_wait_bounded(done, 0);
  if (!ok) {
    s_abort = 1;
    atomicOr(err, kErrWaitTimeout);
  }
  tc_fence_after();
  if (ok && !s_abort && nk > 0) {
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
      const int m = m0 + mt * kTcBM + warp * 32 + lane;
#pragma unroll 1
      for (int cc = 0; cc < BN / CW; ++cc) {
        float v[CW];
        tmem_ld<CW>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * (BN < 32 ? 32 : BN) + cc * CW), v);
        epi.template operator()<CW>(m, n0 + cc * CW, v, (int)blockIdx.z);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (s_abort && threadIdx.x == 0) {
    // drain: the latest copy issued into each stage must land before the CTA exits
    const int issued = s_issued;
    for (int i = issued - kTcStages < 0 ? 0 : issued - kTcStages; i < issued; ++i)
      if (!mbar_wait_bounded(&full[i % kTcStages], (uint32_t)((i / kTcStages) & 1))) atomicOr(err, kErrDrainTimeout);
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

}  // namespace mvsk
