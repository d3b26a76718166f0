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

#include <type_traits>

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

// Bulk tensor stores (shared -> global, bulk-group completion).  The
// coordinates address the tensor map's own dimensions; elements outside its
// extents are not written.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tm, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, const void* src, int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most N bulk groups still reading their shared-memory source
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// every bulk group complete (writes performed)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy shared-memory writes of this thread visible to the async proxy
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

// Epilogues that stage each warp's 32-row x CW-column chunk in shared memory
// (box layout: column-major, the 32 rows contiguous) and write it with one
// bulk tensor store, instead of CW row-scattered stores per thread (a store
// instruction per output line kept a CTA's epilogue at ~10 us).  They define
// kTma = true, kElem (bytes per element), prepare() (CTA-wide set-up in the
// idle operand ring; returns whether it used it), stage() and store().
template <class E, class = void>
struct EpiIsTma : std::false_type {};
template <class E>
struct EpiIsTma<E, std::void_t<decltype(E::kTma)>> : std::bool_constant<E::kTma> {};

// FP32 split-K partials part[(kz*N + n)*ldp + m] through a 3-D tensor map
// {M (stride 4), N (stride 4 ldp), splits (stride 4 N ldp)}, box {32, CW, 1}.
struct EpiPartTma {
  CUtensorMap tm;
  static constexpr bool kTma = true;
  static constexpr int kElem = 4;
  template <int ROWS, int BN>
  __device__ __forceinline__ bool prepare(float*, size_t, int, int) const {
    return false;
  }
  template <int CW, int BN>
  __device__ __forceinline__ void stage(const float (&v)[CW], unsigned char* buf, int lane, int, int, int,
                                        const float*, int, bool) const {
    float* b = reinterpret_cast<float*>(buf);
#pragma unroll
    for (int i = 0; i < CW; ++i) b[i * 32 + lane] = v[i];
  }
  __device__ __forceinline__ void store(const unsigned char* buf, int m, int n, int kz) const {
    tma_store_3d(&tm, buf, m, n, kz);
  }
};

// EpiHvp1 through a 2-D tensor map {T (stride 2), N (stride 2 Tp)} of S^T,
// box {32, CW}; rows T <= t < Tp are outside the map and keep their zeros.
// prepare() puts in shared memory a column table (offset of column c's
// weights, -1 past N) and the CTA's weight block h_q[m0 .. m0 + ROWS) for the
// instances q of its columns, read with batches of independent coalesced
// loads; stage() then reads two shared words per column, without branches.
// When the block does not fit, stage() loads each instance's weight once per
// chunk from global memory.
struct EpiHvp1Tma {
  CUtensorMap tm;
  const float* Hf;
  int T, N, nc;
  static constexpr bool kTma = true;
  static constexpr int kElem = 2;
  template <int ROWS, int BN>
  __device__ __forceinline__ bool prepare(float* ext, size_t cap_floats, int m0, int n0) const {
    const int q0 = n0 / nc, nq = ((n0 + BN < N ? n0 + BN : N) - 1) / nc - q0 + 1;
    if ((size_t)nq * ROWS + BN > cap_floats) return false;
    int* qtab = reinterpret_cast<int*>(ext);
    float* hs = ext + BN;
    for (int c = threadIdx.x; c < BN; c += blockDim.x)
      qtab[c] = n0 + c < N ? ((n0 + c) / nc - q0) * ROWS : -1;
    const float* __restrict__ h = Hf;
    const int tot = nq * ROWS;
    constexpr int kB = 16;
#pragma unroll 1
    for (int base = threadIdx.x; base < tot; base += kB * 128) {
      float r[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int idx = base + u * 128, qi = idx / ROWS, m = m0 + (idx - qi * ROWS);
        r[u] = (idx < tot && m < T) ? __ldg(h + (size_t)(q0 + qi) * T + m) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kB; ++u)
        if (base + u * 128 < tot) hs[base + u * 128] = r[u];
    }
    return true;
  }
  template <int CW, int BN>
  __device__ __forceinline__ void stage(const float (&v)[CW], unsigned char* buf, int lane, int m, int n0, int c0,
                                        const float* ext, int r, bool use) const {
    // every weight of the chunk is read before the first staging store: the
    // stores could alias the weight reads, so interleaving them would chain
    // each read behind the previous store (~15 us per launch)
    float w[CW];
    if (use) {
      const int* __restrict__ qtab = reinterpret_cast<const int*>(ext) + c0;
      const float* __restrict__ hs = ext + BN + r;
#pragma unroll
      for (int i = 0; i < CW; ++i) {
        const int o = qtab[i];
        w[i] = o >= 0 ? hs[o] : 0.f;
      }
    } else {
      const float* __restrict__ h = Hf;
      const bool row = m < T;
      int q = n0 / nc, j = n0 - q * nc;
      float hq = (row && n0 < N) ? __ldg(h + (size_t)q * T + m) : 0.f;
#pragma unroll
      for (int i = 0; i < CW; ++i) {
        w[i] = hq;
        if (++j == nc) {
          j = 0;
          ++q;
          if (i + 1 < CW) hq = (row && n0 + i + 1 < N) ? __ldg(h + (size_t)q * T + m) : 0.f;
        }
      }
    }
    __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(buf);
#pragma unroll
    for (int i = 0; i < CW; ++i) b[i * 32 + lane] = __float2bfloat16(w[i] * v[i]);
  }
  __device__ __forceinline__ void store(const unsigned char* buf, int m, int n, int) const {
    tma_store_2d(&tm, buf, m, n);
  }
};

// Split-K: CTA (x, y, z) computes output tile (n0 = x*BN, m0 = y*128*MT) over the
// k-tiles [z*ktps, min(nk, (z+1)*ktps)) and hands the epilogue its z.  MT = 2
// stacks two 128-row subtiles that share each B tile (accumulators at TMEM
// columns 0 and BN): a third fewer operand bytes per MAC than MT = 1.
// rt (nullable, device): extents known only when the kernel runs (products
// restricted to a face that changes every iteration): rt[0] rows (<= M),
// rt[1] K (<= K), rt[2] split count (every split non-empty), rt[3] k-tiles
// per split; the grid covers the largest values and CTAs outside the runtime
// extents return before any set-up.
template <int BN, int STAGES, class Epi, int MT = 1>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                                                    int ktps, const __grid_constant__ Epi epi, int* err,
                                                    const int* skip, const int* live, const int* rt = nullptr) {
  static_assert(BN == 16 || BN == 32 || BN == 64 || BN == 128 || BN == 192 || BN == 256, "unsupported N tile");
  static_assert(MT == 1 || (MT == 2 && BN >= 32), "two subtiles need BN >= 32");
  constexpr int kTcStages = STAGES;
  constexpr uint32_t TUSED = MT * (BN < 32 ? 32 : BN);
  constexpr uint32_t TCOLS = TUSED <= 32 ? 32 : TUSED <= 64 ? 64 : TUSED <= 128 ? 128 : TUSED <= 256 ? 256 : 512;
  constexpr int CW = BN < 32 ? BN : 32;
  if (skip != nullptr && *skip != 0) return;
  if (live != nullptr && *live == 0) return;
  if (rt != nullptr) {
    const int mr = rt[0], kr = rt[1];
    if (mr < M) M = mr;
    if (kr < K) K = kr;
    ktps = rt[3] > 0 ? rt[3] : 1;
    if ((int)blockIdx.y * kTcBM * MT >= M) return;      // rows beyond the runtime extent
    if ((int)blockIdx.z >= rt[2]) return;               // splits beyond the runtime count
  }
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
  if constexpr (EpiIsTma<Epi>::value) {
    // staging in the operand ring, idle once every MMA has completed: kNBuf
    // buffers per warp, reused after their store has read them; the rest of
    // the ring is the epilogue's prepare() area.
    constexpr int kSB = 32 * CW * Epi::kElem, kNBuf = 4;
    constexpr size_t kRing = (size_t)kTcStages * (ABYTES + BBYTES), kStg = (size_t)4 * kNBuf * kSB;
    static_assert(kStg <= kRing, "staging exceeds the operand ring");
    if (__syncthreads_and(ok && !s_abort && nk > 0)) {
      float* ext = reinterpret_cast<float*>(sm + kStg);
      const bool use = epi.template prepare<MT * kTcBM, BN>(ext, (kRing - kStg) / 4, m0, n0);
      __syncthreads();
      unsigned char* stg = sm + (size_t)warp * kNBuf * kSB;
      int nb = 0;
#pragma unroll 1
      for (int mt = 0; mt < MT; ++mt) {
        const int mrow = m0 + mt * kTcBM + warp * 32;
#pragma unroll 1
        for (int cc = 0; cc < BN / CW; ++cc) {
          const int nn = n0 + cc * CW;
          if (mrow >= M || nn >= N) continue;  // warp-uniform: nothing of this chunk is in the output
          float v[CW];
          tmem_ld<CW>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * (BN < 32 ? 32 : BN) + cc * CW), v);
          unsigned char* buf = stg + (size_t)(nb % kNBuf) * kSB;
          if (nb >= kNBuf) {
            if (lane == 0) bulk_wait_read<kNBuf - 1>();
            __syncwarp();
          }
          epi.template stage<CW, BN>(v, buf, lane, mrow + lane, nn, cc * CW, ext, mt * kTcBM + warp * 32 + lane, use);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            epi.store(buf, mrow, nn, (int)blockIdx.z);
            bulk_commit();
          }
          ++nb;
        }
      }
      if (lane == 0) bulk_wait_all();
      __syncwarp();
    }
  } else if (ok && !s_abort && nk > 0) {
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
