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
// by one unit.  Levels s + u >= 7 are dropped.  Each CTA folds its levels into
// one 64-bit integer per output (sum_l L_l 2^(7(5-l)) + rint(L_6 / 2^7)), and
// a finishing kernel sums the k-splits in integers and scales by
// 2^(e_row + f_col - 49) once, in FP64.  The result is the exact product of
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
constexpr int kOzKc = 512;       // k-values per CTA (exact FP32 accumulation bound)
constexpr int kOzMaxB = 64;      // right-hand vectors per product
constexpr int kOzAStages = 6;    // left-digit tiles in flight (16 KB each)
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

// The kOzS digits of v * 2^-e (|v| < 2^e) as BF16, written plane-strided.
__device__ __forceinline__ void oz_digits(double v, int e, __nv_bfloat16* out, size_t plane) {
  long long R = __double2ll_rn(ldexp(v, kOzExp - e));  // |R| <= 2^49
#pragma unroll
  for (int s = 0; s < kOzS; ++s) {
    const int sh = kOzBits * (kOzS - 1 - s);
    const long long q = sh > 0 ? ((R + (1LL << (sh - 1))) >> sh) : R;  // nearest, ties up
    R -= q * (1LL << sh);
    out[(size_t)s * plane] = __float2bfloat16_rn((float)q);
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
static __global__ void k_oz_col_exp(const double* A, long long lda, long long M, int N, int* e, int Np) {
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

// Right-hand vectors: vector b (b < B) is V[b*vstride + k], k < K.  Exponent
// pass: f[b] = max over chunks of the chunk exponent (f preset to kOzNoExp by
// the caller; all-zero chunks leave it).  Grid (chunks of 1024, Bp).
constexpr int kOzNoExp = (int)0x80808080;  // byte-fill 0x80: below every exponent
static __global__ void __launch_bounds__(256) k_oz_vec_exp(const double* V, long long vstride, int B, int K, int* f,
                                                           const int* need) {
  if (need != nullptr && *need == 0) return;
  const int b = blockIdx.y;
  if (b >= B) return;
  const double* v = V + (size_t)b * vstride;
  double mx = 0.0;
  for (int k = blockIdx.x * 1024 + threadIdx.x; k < K && k < (blockIdx.x + 1) * 1024; k += blockDim.x)
    mx = fmax(mx, fabs(v[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(&f[b], oz_exponent(mx));
}

// Digit pass: rows u*Bp + b of out (ldo BF16 each), zero for k >= K, b >= B or
// an all-zero vector.  Grid (ldo / 256, Bp).
static __global__ void k_oz_vec_digits(const double* V, long long vstride, int B, int Bp, int K, int ldo,
                                       const int* f, __nv_bfloat16* out, const int* need) {
  if (need != nullptr && *need == 0) return;
  const int b = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ldo) return;
  const int e = b < B ? f[b] : kOzNoExp;
  const double x = (e != kOzNoExp && k < K) ? V[(size_t)b * vstride + k] : 0.0;
  oz_digits(x, e != kOzNoExp ? e : 0, out + (size_t)b * ldo + k, (size_t)Bp * ldo);
}

// ------------------------------------------------------------------ product
// part[(z*Bp + b)*ldp + m] = folded levels of sum_{k in split z} A[m,k] V_b[k]
// in units of 2^(e_m + f_b - 49).  Grid (Mp/128, splits); 128 threads.
template <int BP>
__global__ void __launch_bounds__(128, 1) k_oz_gemm(const __nv_bfloat16* __restrict__ Ad,
                                                    const __grid_constant__ CUtensorMap tmX, long long Mp, long long M,
                                                    int K, int nkt, long long* part, long long ldp, int* err,
                                                    const int* need, const int* kinfo = nullptr) {
  static_assert(BP % 16 == 0 && BP <= kOzMaxB, "vector count must be a multiple of 16, at most 64");
  constexpr int NL = kOzS * BP;                        // TMEM columns in use
  constexpr uint32_t TCOLS = NL <= 32 ? 32 : NL <= 64 ? 64 : NL <= 128 ? 128 : NL <= 256 ? 256 : 512;
  constexpr int ABYTES = kTcBM * kTcBK * 2;            // one left digit tile
  constexpr int XBYTES = kOzS * BP * kTcBK * 2;        // all right digits of one k-block
  if (need != nullptr && *need == 0) return;
  if (kinfo != nullptr) {  // left operand restricted to a coordinate list: K = its padded count
    K = kinfo[1];
    nkt = K / kTcBK;
    if ((int)blockIdx.y * (kOzKc / kTcBK) >= nkt) return;  // k-chunks beyond the runtime K
  }
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sX = sm;
  unsigned char* sA = sm + (size_t)kOzXStages * XBYTES;
  uint64_t* xfull = reinterpret_cast<uint64_t*>(sA + (size_t)kOzAStages * ABYTES);
  uint64_t* xempty = xfull + kOzXStages;
  uint64_t* afull = xempty + kOzXStages;
  uint64_t* aempty = afull + kOzAStages;
  uint64_t* done = aempty + kOzAStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int s_abort;
  __shared__ int s_xissued, s_aissued;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long m0 = (long long)blockIdx.x * kTcBM;
  const int nkb = (K + kTcBK - 1) / kTcBK;
  const int kb0 = blockIdx.y * (kOzKc / kTcBK);
  const int kb1 = kb0 + kOzKc / kTcBK < nkb ? kb0 + kOzKc / kTcBK : nkb;
  const int nk = kb1 > kb0 ? kb1 - kb0 : 0;
  if (threadIdx.x == 0) {
    s_abort = 0;
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
    mbar_init(done, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    int ai = 0;
    for (int i = 0; i < nk && !s_abort; ++i) {
      const int xs = i % kOzXStages;
      if (i >= kOzXStages && !mbar_wait_bounded(&xempty[xs], (uint32_t)(((i / kOzXStages) - 1) & 1))) {
        s_abort = 1;
        atomicOr(err, kErrWaitTimeout);
        break;
      }
      mbar_expect_tx(&xfull[xs], XBYTES);
#pragma unroll 1
      for (int u = 0; u < kOzS; ++u)
        tma_load_2d(sX + (size_t)xs * XBYTES + (size_t)u * BP * 128, &tmX, (kb0 + i) * kTcBK, u * BP, &xfull[xs]);
      s_xissued = i + 1;
#pragma unroll 1
      for (int s = 0; s < kOzS; ++s, ++ai) {
        const int as = ai % kOzAStages;
        if (ai >= kOzAStages && !mbar_wait_bounded(&aempty[as], (uint32_t)(((ai / kOzAStages) - 1) & 1))) {
          s_abort = 1;
          atomicOr(err, kErrWaitTimeout);
          break;
        }
        mbar_expect_tx(&afull[as], ABYTES);
        bulk_g2s(sA + (size_t)as * ABYTES,
                 Ad + (size_t)s * Mp * nkt * 64 + ((size_t)blockIdx.x * nkt + (size_t)(kb0 + i)) * 8192, ABYTES,
                 &afull[as]);
        s_aissued = ai + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    int ai = 0;
    for (int i = 0; i < nk && !s_abort; ++i) {
      const int xs = i % kOzXStages;
      if (!mbar_wait_bounded(&xfull[xs], (uint32_t)((i / kOzXStages) & 1))) {
        s_abort = 1;
        atomicOr(err, kErrWaitTimeout);
        break;
      }
      tc_fence_after();
      const unsigned char* xb = sX + (size_t)xs * XBYTES;
      bool ok = true;
#pragma unroll 1
      for (int s = 0; s < kOzS; ++s, ++ai) {
        const int as = ai % kOzAStages;
        if (!mbar_wait_bounded(&afull[as], (uint32_t)((ai / kOzAStages) & 1))) {
          s_abort = 1;
          atomicOr(err, kErrWaitTimeout);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t da = umma_desc_sw128(sA + (size_t)as * ABYTES);
        const int ntot = (kOzS - s) * BP;
#pragma unroll
        for (int kk = 0; kk < kTcBK / 16; ++kk) {
          const uint32_t acc = (i > 0 || s > 0 || kk > 0) ? 1u : 0u;
#pragma unroll 1
          for (int c0 = 0; c0 < ntot; c0 += 256) {
            const int nn = ntot - c0 < 256 ? ntot - c0 : 256;
            const uint64_t db = umma_desc_sw128(xb + (size_t)c0 * 128);
            umma_bf16(tmem + (uint32_t)(s * BP + c0), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk),
                      idesc_bf16_f32(kTcBM, nn), acc);
          }
        }
        umma_commit(&aempty[as]);
      }
      if (!ok) break;
      umma_commit(&xempty[xs]);
    }
    umma_commit(done);  // arrives once every MMA issued above has completed
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(done, 0);
  if (!ok) {
    s_abort = 1;
    atomicOr(err, kErrWaitTimeout);
  }
  tc_fence_after();
  if (ok && !s_abort) {
    const long long m = m0 + warp * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int b0 = 0; b0 < BP; b0 += 16) {
      long long acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = 0;
      if (nk > 0) {
        // Integer values of the FP32 levels by FP32/INT arithmetic only (a
        // float-to-int64 conversion runs on the FP64 pipe): for |w| < 2^22,
        // w + 1.5*2^23 rounds w to the nearest integer in the low mantissa bits.
        constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
        constexpr int kMagicBits = 0x4B400000;
#pragma unroll 1
        for (int l = 0; l < kOzS; ++l) {
          float v[16];
          tmem_ld16(lane_base + (uint32_t)(l * BP + b0), v);
          if (l < kOzS - 1) {  // exact integer, |v| <= 2^24: v = 4096 hi + lo
            const int sh = kOzBits * (kOzS - 2 - l);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const float t = fmaf(v[q], 1.0f / 4096.0f, kMagic);
              const int hi = __float_as_int(t) - kMagicBits;
              const float lo = fmaf(-(t - kMagic), 4096.0f, v[q]);
              const int il = __float_as_int(lo + kMagic) - kMagicBits;
              acc[q] += (long long)hi * (1LL << (sh + 12)) + (long long)il * (1LL << sh);
            }
          } else {  // level kOzS-1 in units of 2^kOzBits of it, rounded
#pragma unroll
            for (int q = 0; q < 16; ++q)
              acc[q] += __float_as_int(fmaf(v[q], 1.0f / (float)(1 << kOzBits), kMagic)) - kMagicBits;
          }
        }
      }
      if (m < M) {
#pragma unroll
        for (int q = 0; q < 16; ++q) part[((size_t)blockIdx.y * BP + b0 + q) * ldp + m] = acc[q];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (s_abort && threadIdx.x == 0) {
    // drain: the latest copies issued into each stage must land before the CTA exits
    const int xi = s_xissued, ai = s_aissued;
    for (int i = xi - kOzXStages < 0 ? 0 : xi - kOzXStages; i < xi; ++i)
      if (!mbar_wait_bounded(&xfull[i % kOzXStages], (uint32_t)((i / kOzXStages) & 1))) atomicOr(err, kErrDrainTimeout);
    for (int i = ai - kOzAStages < 0 ? 0 : ai - kOzAStages; i < ai; ++i)
      if (!mbar_wait_bounded(&afull[i % kOzAStages], (uint32_t)((i / kOzAStages) & 1))) atomicOr(err, kErrDrainTimeout);
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

// Sum of the split partials of output (m, b) scaled to its FP64 value.
__device__ __forceinline__ double oz_value(const long long* part, int splits, int Bp, long long ldp, long long m, int b,
                                           int em, int fb) {
  double v = 0.0;
  for (int z0 = 0; z0 < splits; z0 += 16) {
    long long s = 0;  // at most 16 partials of magnitude < 2^58.1: no overflow
    const int z1 = z0 + 16 < splits ? z0 + 16 : splits;
#pragma unroll 4
    for (int z = z0; z < z1; ++z) s += part[((size_t)z * Bp + b) * ldp + m];
    v += (double)s;
  }
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
