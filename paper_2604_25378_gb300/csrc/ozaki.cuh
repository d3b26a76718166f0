// FP64-accurate products A V and A^T V on the BF16 tensor cores.
//
// Ozaki's error-free splitting (Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), run on
// tensor cores with FP32 accumulation as in Mukunoki, Ozaki, Ogita, Imamura
// ("DGEMM using Tensor Cores, and Its Accurate and Reproducible Versions",
// ISC 2020).  On this part the FP64 pipe delivers about 2 FMA/clk/SM; the
// split product runs on the BF16 tensor pipe instead.
//
// Splitting.  Every row of the left operand and every column vector of the
// right operand is scaled by a power of two so that |.| < 1, rounded to a
// 49-bit fixed-point integer R and cut into kOzS = 7 balanced base-128 digits
//     value = 2^e * sum_s q_s 2^(-7(s+1)),  |q_0| <= 128, |q_s| <= 64 (s > 0),
// each q_s exactly representable in BF16.  A digit product is an integer of
// magnitude <= 2^14; products with s + u = l (level l) share one FP32 TMEM
// accumulator.  Over kOzKc = 512 k-values every level l <= 5 stays within
// 2^24 and is accumulated exactly; level 6 (weight 2^-42 of level 0) may round
// by one unit.  Levels s + u >= 7 are dropped.  The levels of every 512-value
// chunk are folded into one 64-bit integer per output (sum_l L_l 2^(7(5-l)) +
// rint(L_6 / 2^7)), chunks are summed in integers (slots of 16 chunks), and a
// finishing kernel adds the slots and scales by 2^(e_row + f_col - 49) once,
// in FP64.  The result is the exact product of
// the 49-bit roundings of both operands, up to the dropped levels.
//
// GEMM layout.  Left operand: kOzS digit planes, each Mp x ldk BF16 stored as
// contiguous 128 x 64 tiles (row tile, then k tile) whose bytes are already in
// the 128-byte-swizzled order the MMA reads from shared memory, so that one
// 16 KB bulk copy moves a tile (sequential DRAM reads instead of 128 strided
// 128-byte rows).  Right operand: the
// digit planes of Bp <= 64 vectors stacked as rows u*Bp + b (ldk BF16 each).
// TMEM columns [l*Bp, (l+1)*Bp) hold level l; the MMA of left digit s takes
// the right digits u = 0..kOzS-1-s as one N = (kOzS-s)*Bp operand and writes
// at column s*Bp, so block u lands on level s+u.
#pragma once

#include "gemm_tc.cuh"

namespace mvsk {

constexpr int kOzS = 7;          // digits per operand
constexpr int kOzBits = 7;       // bits per digit
constexpr int kOzKc = 512;       // k-values per TMEM accumulation (exact FP32 bound)
constexpr int kOzMaxB = 64;      // right-hand vectors per product
constexpr int kOzAStages = 7;    // left-digit tiles in flight (16 KB each)
constexpr int kOzXStages = 2;    // right-digit k-blocks in flight (kOzS*Bp*128 bytes each)
constexpr int kOzExp = kOzS * kOzBits;  // 49: fixed-point bits of one operand

__host__ __device__ constexpr size_t oz_smem_bytes(int Bp) {
  return 1024 + (size_t)kOzXStages * kOzS * Bp * 128 + (size_t)kOzAStages * kTcBM * kTcBK * 2 + 256;
}

// Element offset of (row r, column k) in a plane of 128 x 64 tiles with nkt
// k-tiles per row tile: 16-byte chunk j of row r sits at chunk j ^ (r mod 8).
__host__ __device__ __forceinline__ size_t oz_tiled(long long r, int k, int nkt) {
  const int rr = (int)(r & 127), kk = k & 63;
  return ((size_t)(r >> 7) * nkt + (k >> 6)) * 8192 + (size_t)rr * 64 + (size_t)((((kk >> 3) ^ (rr & 7)) << 3) | (kk & 7));
}

// Exponent e with |v| < 2^e for every |v| <= vmax (0 for vmax = 0).
__device__ __forceinline__ int oz_exponent(double vmax) {
  int e = 0;
  if (vmax > 0.0 && isfinite(vmax)) frexp(vmax, &e);
  return e;
}

// R = round(v * 2^(kOzExp - e)) (nearest, ties to even) for |v| < 2^e, from
// the bits of v with integer operations only: an FP64 scaling and conversion
// would take the FP64 pipe (about 2 operations/clk/SM on this part).  The
// mantissa m (implicit bit included) times 2^(E - 1075) is shifted right by
// k = 1075 - E - kOzExp + e places (k >= 4 for normal v, |v| < 2^e; a
// subnormal v may take a left shift).  0 for k >= 64 and for non-finite v.
__device__ __forceinline__ long long oz_fixed(double v, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0x7FF) return 0;
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (E != 0 ? (1ull << 52) : 0ull);
  const int k = (E != 0 ? 1075 - E : 1074) - kOzExp + e;
  if (k >= 64 || m == 0) return 0;
  unsigned long long q;
  if (k <= 0) {
    q = m << (-k);  // subnormal v with e <= -1025: exact (q < 2^49 by the contract)
  } else {
    q = m >> k;
    const unsigned long long rem = m & ((1ull << k) - 1ull), half = 1ull << (k - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  return (bits >> 63) ? -(long long)q : (long long)q;
}

// The kOzS digits of v * 2^-e (|v| < 2^e) as BF16, written plane-strided.
// Digit values |q| <= 128 are exact in FP32 and BF16; the FP32 value comes
// from the integer by the 1.5 * 2^23 offset (FP32 pipe, no conversion unit).
__device__ __forceinline__ void oz_digits(double v, int e, __nv_bfloat16* out, size_t plane) {
  long long R = oz_fixed(v, e);  // |R| <= 2^49
#pragma unroll
  for (int s = 0; s < kOzS; ++s) {
    const int sh = kOzBits * (kOzS - 1 - s);
    const long long q = sh > 0 ? ((R + (1LL << (sh - 1))) >> sh) : R;  // nearest, ties up
    R -= q * (1LL << sh);
    const float qf = __int_as_float(0x4B400000 + (int)q) - 12582912.0f;
    out[(size_t)s * plane] = __float2bfloat16_rn(qf);
  }
}

// ------------------------------------------------------------ operand prep
// e[m] for the rows of a row-major M x K FP64 matrix (one warp per row).
static __global__ void k_oz_row_exp(const double* A, long long lda, long long M, int K, int* e, long long Mp) {
  const long long m = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (m >= Mp) return;
  double mx = 0.0;
  if (m < M)
    for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(A[(size_t)m * lda + k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) e[m] = oz_exponent(mx);
}

// e[j] for the columns j < N of a row-major M x N FP64 matrix (zero for N <= j < Np).
// Block (32, 32): 32 columns, rows strided over threadIdx.y.
static __global__ void __launch_bounds__(1024) k_oz_col_exp(const double* A, long long lda, long long M, int N, int* e, int Np) {
  __shared__ double red[32][33];
  const int j = blockIdx.x * 32 + threadIdx.x;
  double mx = 0.0;
  if (j < N)
    for (long long m = threadIdx.y; m < M; m += 32) mx = fmax(mx, fabs(A[(size_t)m * lda + j]));
  red[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0) {
    for (int q = 1; q < 32; ++q) mx = fmax(mx, red[q][threadIdx.x]);
    if (j < Np) e[j] = oz_exponent(mx);
  }
}

// Digit planes of the rows (tiled, plane = Mp*ldo elements), zero for m >= M or k >= K.
static __global__ void k_oz_split_rows(const double* A, long long lda, long long M, int K, const int* e,
                                       __nv_bfloat16* out, long long Mp, int ldo) {
  const size_t plane = (size_t)Mp * ldo;
  const int nkt = ldo / 64;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    const long long m = (long long)(i / ldo);
    const int k = (int)(i % ldo);
    const double v = (m < M && k < K) ? A[(size_t)m * lda + k] : 0.0;
    oz_digits(v, e[m], out + oz_tiled(m, k, nkt), plane);
  }
}

// Digit planes of the columns (transposed, tiled): digits of A[m][j] at row j,
// column m, with exponent e[j] (plane = Np*ldo), zero for j >= N or m >= M.
static __global__ void k_oz_split_cols(const double* A, long long lda, long long M, int N, const int* e,
                                       __nv_bfloat16* out, int Np, long long ldo) {
  __shared__ double tile[32][33];
  const long long m0 = (long long)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long long m = m0 + threadIdx.y + 8 * q;
    const int j = j0 + threadIdx.x;
    tile[threadIdx.y + 8 * q][threadIdx.x] = (m < M && j < N) ? A[(size_t)m * lda + j] : 0.0;
  }
  __syncthreads();
  const size_t plane = (size_t)Np * ldo;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = j0 + threadIdx.y + 8 * q;
    const long long m = m0 + threadIdx.x;
    if (j < Np && m < ldo) oz_digits(tile[threadIdx.x][threadIdx.y + 8 * q], e[j], out + oz_tiled(j, (int)m, (int)(ldo / 64)), plane);
  }
}

// Digit planes of the columns of A in a coordinate list (idx[j], j < info[0];
// zero up to the padded count info[1], a multiple of 64) in the same tiled
// layout with nkt = info[1] / 64 k-tiles and plane stride Mp * info[1]; the
// exponents e[m] of the full rows bound every selected entry.
static __global__ void k_oz_split_rows_u(const double* A, long long lda, long long M, const int* idx, const int* info,
                                         const int* e, __nv_bfloat16* out, long long Mp) {
  const int ku = info[0], kup = info[1];
  const size_t plane = (size_t)Mp * kup;
  const int nkt = kup / 64;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    const long long m = (long long)(i / kup);
    const int k = (int)(i % kup);
    const double v = (m < M && k < ku) ? A[(size_t)m * lda + idx[k]] : 0.0;
    oz_digits(v, e[m], out + oz_tiled(m, k, nkt), plane);
  }
}

// Right-hand vectors, one launch per product: vector b < B has elements
// v_k = V[b*vstride + k] for k < K (gidx null) or v_k = V[b*vstride + gidx[k]]
// for k < ginfo[0] (a gathered coordinate list), zero up to the row length
// ldo (ginfo[1] when gathered); vectors B <= b < Bp are zero.  CTA (x, b)
// finds the exponent of vector b from the largest magnitude, taken as the
// largest bit pattern of |v_k| (integer pipe; the order of non-negative
// doubles), and writes the digits of its share of the row: rows u*Bp + b of
// out (ldo BF16 each).  CTA (0, b) stores f[b] (kOzNoExp for a zero or absent
// vector).  The zn int64 slots at zp are zeroed over the whole grid (the
// product's integer slots).  Grid (chunks, Bp), 512 threads.
constexpr int kOzNoExp = (int)0x80808080;  // byte-fill 0x80: below every exponent
static __global__ void __launch_bounds__(512) k_oz_vec_split(const double* V, long long vstride, int B, int K, int ldo,
                                                             const int* gidx, const int* ginfo, int* f,
                                                             __nv_bfloat16* out, int Bp, long long* zp, long long zn,
                                                             const int* need) {
  if (need != nullptr && *need == 0) return;
  const int b = blockIdx.y;
  const long long nth = (long long)gridDim.x * gridDim.y * blockDim.x;
  for (long long i = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x; i < zn; i += nth)
    zp[i] = 0;
  const int kv = gidx != nullptr ? ginfo[0] : K;     // elements that may be nonzero
  const int row = gidx != nullptr ? ginfo[1] : ldo;  // digits written (the product reads no further)
  const double* v = V + (size_t)(b < B ? b : 0) * vstride;
  __shared__ unsigned long long wm[16];
  __shared__ int s_e;
  unsigned long long mx = 0;
  if (b < B)
    for (int k = threadIdx.x; k < kv; k += blockDim.x) {
      const double x = gidx != nullptr ? v[gidx[k]] : v[k];
      const unsigned long long m = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
      mx = m > mx ? m : mx;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = wm[w] > m ? wm[w] : m;
    const int e = m != 0 ? oz_exponent(__longlong_as_double((long long)m)) : kOzNoExp;
    s_e = e;
    if (blockIdx.x == 0) f[b] = e;
  }
  __syncthreads();
  const int e = s_e;
  const int chunk = (row + (int)gridDim.x - 1) / (int)gridDim.x;
  const int k0 = (int)blockIdx.x * chunk, k1 = k0 + chunk < row ? k0 + chunk : row;
  for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) {
    double x = 0.0;
    if (e != kOzNoExp && k < kv) x = gidx != nullptr ? v[gidx[k]] : v[k];
    oz_digits(x, e != kOzNoExp ? e : 0, out + (size_t)b * ldo + k, (size_t)Bp * ldo);
  }
}

// CTAs per vector of k_oz_vec_split for rows of ldo digits.
inline int oz_split_chunks(long long ldo) {
  const long long s = (ldo + 2047) / 2048;
  return (int)(s < 1 ? 1 : s > 8 ? 8 : s);
}

// ------------------------------------------------------------------ product
// Persistent split product.  Work units are (row tile mt, k-chunk ch): the
// 128 rows of tile mt against the <= 8 k-blocks (512 k-values) of chunk ch,
// U = (Mp / 128) * nch of them, ordered row-tile-major; CTA c of the G in the
// grid takes units [c U / G, (c + 1) U / G).  Per unit the MMAs accumulate
// the seven levels in TMEM (exact, as above), and the epilogue warps fold
// them into 64-bit integers held in registers across the CTA's consecutive
// units of one row tile and one group of kOzGroup chunks; at a change of
// either (or the end of the range) the group sum goes to slot g = ch /
// kOzGroup by 64-bit integer atomic addition, so that
//     part[(g*Bp + b)*ldp + m] = sum over chunks of group g of the chunk's folded levels
// whatever the order of the additions (integer sums are associative).  The
// slots must be zero before the launch (k_oz_vec_split clears them).  Each chunk's sum is
// < 2^58.1 in magnitude, so a slot of 16 stays below 2^62.1.
//
// Roles: warp 0 streams the operands (one bulk copy per 16 KB left digit
// tile, one TMA box per right digit block of a k-block), warp 1 issues the
// MMAs, and kOzEpiWarps warps drain TMEM (four per TMEM lane quarter, 16
// columns of each level apiece).  TMEM holds one unit: the MMAs of the next
// unit wait until every epilogue warp has read the levels (tmem_empty), while
// the loads run ahead through the shared-memory ring; the integer atomics of
// a finished group overlap the next unit's MMAs.  Grid: at most one CTA per
// SM (about 225 KB of shared memory), kOzThreads threads.
constexpr int kOzEpiWarps = 16;
constexpr int kOzThreads = 64 + 32 * kOzEpiWarps;
constexpr int kOzGroup = 16;  // chunks per integer slot

// Integer slots of a product over nkb k-blocks.
__host__ __device__ constexpr int oz_slots(int nkb) { return ((nkb + 7) / 8 + kOzGroup - 1) / kOzGroup; }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// kinfo (nullable): the left operand is restricted to a coordinate list whose
// padded length kinfo[1] (a multiple of 64) replaces K.
template <int BP>
__global__ void __launch_bounds__(kOzThreads, 1) k_oz_gemm(const __nv_bfloat16* __restrict__ Ad,
                                                           const __grid_constant__ CUtensorMap tmX, long long Mp,
                                                           long long M, int K, int nkt, long long* part, long long ldp,
                                                           int* err, const int* need, const int* kinfo = nullptr) {
  static_assert(BP % 16 == 0 && BP <= kOzMaxB, "vector count must be a multiple of 16, at most 64");
  constexpr int NL = kOzS * BP;                        // TMEM columns in use
  constexpr uint32_t TCOLS = NL <= 32 ? 32 : NL <= 64 ? 64 : NL <= 128 ? 128 : NL <= 256 ? 256 : 512;
  constexpr int ABYTES = kTcBM * kTcBK * 2;            // one left digit tile
  constexpr int XBYTES = kOzS * BP * kTcBK * 2;        // all right digits of one k-block
  constexpr int NSL = BP / 16;                         // 16-column slices of a level
  if (need != nullptr && *need == 0) return;
  if (kinfo != nullptr) {
    K = kinfo[1];
    nkt = K / kTcBK;
  }
  const int nkb = (K + kTcBK - 1) / kTcBK;
  const int nch = (nkb + 7) / 8;
  const long long U = (Mp / kTcBM) * (long long)nch;
  const long long u0 = (long long)blockIdx.x * U / gridDim.x, u1 = (long long)(blockIdx.x + 1) * U / gridDim.x;
  if (u0 >= u1) return;  // uniform over the CTA: before any barrier or TMEM use

  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sX = sm;
  unsigned char* sA = sm + (size_t)kOzXStages * XBYTES;
  uint64_t* xfull = reinterpret_cast<uint64_t*>(sA + (size_t)kOzAStages * ABYTES);
  uint64_t* xempty = xfull + kOzXStages;
  uint64_t* afull = xempty + kOzXStages;
  uint64_t* aempty = afull + kOzAStages;
  uint64_t* tfull = aempty + kOzAStages;  // a unit's levels are in TMEM
  uint64_t* tempty = tfull + 1;           // every epilogue warp has read them
  uint64_t* mdone = tempty + 1;           // every MMA issued has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  __shared__ int s_abort_raw, s_xissued, s_aissued;
  volatile int* s_abort = &s_abort_raw;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    *s_abort = 0;
    s_xissued = 0;
    s_aissued = 0;
    for (int s = 0; s < kOzXStages; ++s) {
      mbar_init(&xfull[s], 1);
      mbar_init(&xempty[s], 1);
    }
    for (int s = 0; s < kOzAStages; ++s) {
      mbar_init(&afull[s], 1);
      mbar_init(&aempty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, kOzEpiWarps);
    mbar_init(mdone, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // producer
      int i = 0, ai = 0;
      bool ok = true;
      for (long long u = u0; u < u1 && ok; ++u) {
        const long long mt = u / nch;
        const int kb0 = (int)(u % nch) * 8, kb1 = kb0 + 8 < nkb ? kb0 + 8 : nkb;
        for (int kb = kb0; kb < kb1 && ok; ++kb, ++i) {
          const int xs = i % kOzXStages;
          if (*s_abort || (i >= kOzXStages && !mbar_wait_bounded(&xempty[xs], (uint32_t)(((i / kOzXStages) - 1) & 1)))) {
            ok = false;
            break;
          }
          mbar_expect_tx(&xfull[xs], XBYTES);
#pragma unroll 1
          for (int v = 0; v < kOzS; ++v)
            tma_load_2d(sX + (size_t)xs * XBYTES + (size_t)v * BP * 128, &tmX, kb * kTcBK, v * BP, &xfull[xs]);
          s_xissued = i + 1;
#pragma unroll 1
          for (int s = 0; s < kOzS; ++s, ++ai) {
            const int as = ai % kOzAStages;
            if (ai >= kOzAStages && !mbar_wait_bounded(&aempty[as], (uint32_t)(((ai / kOzAStages) - 1) & 1))) {
              ok = false;
              break;
            }
            mbar_expect_tx(&afull[as], ABYTES);
            bulk_g2s(sA + (size_t)as * ABYTES, Ad + (size_t)s * Mp * nkt * 64 + ((size_t)mt * nkt + (size_t)kb) * 8192,
                     ABYTES, &afull[as]);
            s_aissued = ai + 1;
          }
        }
      }
      if (!ok) {
        *s_abort = 1;
        atomicOr(err, kErrWaitTimeout);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issue
      // With as many left-digit slots as digits, tile s of every k-block
      // sits in slot s (filled for k-block i in phase i & 1).  The loops over
      // digits, k-steps and N pieces are unrolled, so that every MMA is one
      // instruction on precomputed descriptors and a constant instruction
      // descriptor: a single thread issues them, and per-MMA bookkeeping
      // would otherwise hold the tensor pipe back on the narrow pieces.
      static_assert(kOzAStages == kOzS && kOzXStages == 2, "slot s holds digit s; two right-digit slots");
      uint64_t adesc[kOzS];
#pragma unroll
      for (int s = 0; s < kOzS; ++s) adesc[s] = umma_desc_sw128(sA + (size_t)s * ABYTES);
      const uint64_t xdesc0 = umma_desc_sw128(sX), xdesc1 = umma_desc_sw128(sX + XBYTES);
      int i = 0, r = 0;
      bool ok = true;
      for (long long u = u0; u < u1 && ok; ++u, ++r) {
        const int kb0 = (int)(u % nch) * 8, kb1 = kb0 + 8 < nkb ? kb0 + 8 : nkb;
        if (r > 0) {
          if (*s_abort || !mbar_wait_bounded(tempty, (uint32_t)((r - 1) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        for (int kb = kb0; kb < kb1 && ok; ++kb, ++i) {
          const int xs = i & 1;
          if (*s_abort || !mbar_wait_bounded(&xfull[xs], (uint32_t)((i >> 1) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t xd = xs ? xdesc1 : xdesc0;
          const uint32_t ph = (uint32_t)(i & 1);
          const bool first = kb == kb0;
#pragma unroll
          for (int s = 0; s < kOzS; ++s) {
            if (!mbar_wait_bounded(&afull[s], ph)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < kTcBK / 16; ++kk) {
              const uint32_t acc = (!first || s > 0 || kk > 0) ? 1u : 0u;
#pragma unroll
              for (int c0 = 0; c0 < (kOzS - s) * BP; c0 += 256) {
                const int nn = (kOzS - s) * BP - c0 < 256 ? (kOzS - s) * BP - c0 : 256;
                umma_bf16(tmem + (uint32_t)(s * BP + c0), adesc[s] + (uint64_t)(2 * kk),
                          xd + (uint64_t)(c0 * 8 + 2 * kk), idesc_bf16_f32(kTcBM, nn), acc);
              }
            }
            umma_commit(&aempty[s]);
          }
          if (ok) umma_commit(&xempty[xs]);
        }
        if (ok) umma_commit(tfull);
      }
      if (!ok) {
        *s_abort = 1;
        atomicOr(err, kErrWaitTimeout);
      }
      umma_commit(mdone);  // arrives once every MMA issued above has completed
      if (!mbar_wait_bounded(mdone, 0)) atomicOr(err, kErrDrainTimeout);
    }
  } else {  // epilogue: TMEM lane quarter q, columns [16 sl, 16 sl + 16) of each level
    const int ew = warp - 2, q = warp & 3, sl = ew >> 2;
    const bool act = sl < NSL;
    const uint32_t lb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(sl * 16);
    long long acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0;
    long long cur_mt = -1;
    int cur_g = -1, r = 0;
    auto flush = [&]() {
      const long long m = cur_mt * kTcBM + q * 32 + lane;
      if (act && m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          atomicAdd(reinterpret_cast<unsigned long long*>(part + ((size_t)cur_g * BP + sl * 16 + j) * ldp + m),
                    (unsigned long long)acc[j]);
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = 0;
    };
    bool ok = true;
    for (long long u = u0; u < u1; ++u, ++r) {
      const long long mt = u / nch;
      const int g = (int)(u % nch) / kOzGroup;
      if (cur_mt >= 0 && (mt != cur_mt || g != cur_g)) flush();
      cur_mt = mt;
      cur_g = g;
      if (*s_abort || !mbar_wait_bounded(tfull, (uint32_t)(r & 1))) {
        ok = false;
        break;
      }
      tc_fence_after();
      if (act) {
        // Integer values of the FP32 levels by FP32/INT arithmetic only (a
        // float-to-int64 conversion runs on the FP64 pipe): for |w| < 2^22,
        // w + 1.5*2^23 rounds w to the nearest integer in the low mantissa bits.
        constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
        constexpr int kMagicBits = 0x4B400000;
#pragma unroll 1
        for (int l = 0; l < kOzS; ++l) {
          float v[16];
          tmem_ld16(lb + (uint32_t)(l * BP), v);
          if (l < kOzS - 1) {  // exact integer, |v| <= 2^24: v = 4096 hi + lo
            const int sh = kOzBits * (kOzS - 2 - l);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float t = fmaf(v[j], 1.0f / 4096.0f, kMagic);
              const int hi = __float_as_int(t) - kMagicBits;
              const float lo = fmaf(-(t - kMagic), 4096.0f, v[j]);
              const int il = __float_as_int(lo + kMagic) - kMagicBits;
              acc[j] += (long long)(hi * 4096 + il) * (1LL << sh);
            }
          } else {  // level kOzS-1 in units of 2^kOzBits of it, rounded
#pragma unroll
            for (int j = 0; j < 16; ++j)
              acc[j] += __float_as_int(fmaf(v[j], 1.0f / (float)(1 << kOzBits), kMagic)) - kMagicBits;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);
    }
    if (ok && cur_mt >= 0) flush();
    if (!ok) {
      if (lane == 0) atomicOr(err, kErrWaitTimeout);
      *s_abort = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*s_abort && threadIdx.x == 0) {
    // drain: the latest copies issued into each stage must land before the CTA exits
    const int xi = s_xissued, ai = s_aissued;
    for (int i = xi - kOzXStages < 0 ? 0 : xi - kOzXStages; i < xi; ++i)
      if (!mbar_wait_bounded(&xfull[i % kOzXStages], (uint32_t)((i / kOzXStages) & 1))) atomicOr(err, kErrDrainTimeout);
    for (int i = ai - kOzAStages < 0 ? 0 : ai - kOzAStages; i < ai; ++i)
      if (!mbar_wait_bounded(&afull[i % kOzAStages], (uint32_t)((i / kOzAStages) & 1))) atomicOr(err, kErrDrainTimeout);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TCOLS);
  }
}

// FP64 value of output (m, b) from its integer slots.
__device__ __forceinline__ double oz_value(const long long* part, int slots, int Bp, long long ldp, long long m, int b,
                                           int em, int fb) {
  double v = 0.0;
  for (int z = 0; z < slots; ++z) v += (double)part[((size_t)z * Bp + b) * ldp + m];
  // digit weights 2^-7(s+1) and 2^-7(u+1), folded levels 2^(7(kOzS-2)):  2^(e + f - 49)
  return fb == kOzNoExp ? 0.0 : ldexp(v, em + fb - kOzExp);
}

// Plain store of the product (the reference entry point and tests):
// out[b*ostride + m] = alpha * (A V_b)[m] for m < M, b < B.
static __global__ void k_oz_store(const long long* part, int splits, int Bp, long long ldp, long long M, int B,
                                  const int* em, const int* fb, double alpha, double* out, long long ostride) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (m >= M || b >= B) return;
  out[(size_t)b * ostride + m] = alpha * oz_value(part, splits, Bp, ldp, m, b, em[m], fb[b]);
}

}  // namespace mvsk
