// Dense FP64 building blocks of the direct configuration: a tiled SIMT GEMM,
// a pivot-block Cholesky/inverse, and the block Gauss-Jordan sweep that
// inverts the face matrix B (SPD iff the reduced tangent Hessian is).
#pragma once

#include "common.cuh"

namespace mvsk {

// C[i*ldc + j] = beta*C + alpha * sum_k opA(i,k) * opB(j,k) * (sk ? sk[k] : 1),
// i < M, j < N, k < K.  opA(i,k) = A[i*lda + k] (AT = false) or A[k*lda + i]
// (AT = true); opB(j,k) = B[j*ldb + k] (BT = false) or B[k*ldb + j] (BT = true).
// 64 x 64 tiles, 16-deep k slices, 256 threads with 4 x 4 outputs each.
template <bool AT, bool BT>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha, const double* __restrict__ A,
                                               long long lda, const double* __restrict__ B, long long ldb,
                                               const double* __restrict__ sk, double beta, double* C,
                                               long long ldc) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    // 64 x 16 elements of each operand, 4 per thread
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * 256;
      int r, kk;
      if (AT) {  // consecutive threads along the M index (contiguous in memory)
        r = e % 64;
        kk = e / 64;
      } else {
        kk = e % 16;
        r = e / 16;
      }
      const int gi = i0 + r, gk = k0 + kk;
      As[kk][r] = (gi < M && gk < K) ? (AT ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk]) : 0.0;
      if (BT) {
        r = e % 64;
        kk = e / 64;
      } else {
        kk = e % 16;
        r = e / 16;
      }
      const int gj = j0 + r, gk2 = k0 + kk;
      double bv = (gj < N && gk2 < K) ? (BT ? B[(size_t)gk2 * ldb + gj] : B[(size_t)gj * ldb + gk2]) : 0.0;
      if (sk != nullptr && gk2 < K) bv *= sk[gk2];
      Bs[kk][r] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty * 4 + q];
        b[q] = Bs[kk][tx * 4 + q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = i0 + ty * 4 + p;
    if (i >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tx * 4 + q;
      if (j >= N) continue;
      double* c = C + (size_t)i * ldc + j;
      *c = (beta == 0.0 ? 0.0 : beta * *c) + alpha * acc[p][q];
    }
  }
}

// Cholesky factor and inverse of the b x b pivot block A[k0.., k0..] (lda):
// P = A_kk^-1 written to P (b x b, ld b).  flag |= 1 when a pivot is not
// positive and finite (block not positive definite).  One CTA, b <= 64.
__global__ void __launch_bounds__(256) k_pivot_inverse(const double* A, long long lda, int k0, int b, double* P,
                                                       int* flag) {
  __shared__ double L[64][65];
  __shared__ double Li[64][65];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < 64 * 64; e += blockDim.x) {
    const int r = e / 64, c = e % 64;
    L[r][c] = (r < b && c < b) ? A[(size_t)(k0 + r) * lda + k0 + c] : 0.0;
    Li[r][c] = 0.0;
  }
  __syncthreads();
  // right-looking Cholesky in shared memory (lower triangle)
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      const double d = L[j][j];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      L[j][j] = sqrt(fmax(d, 1e-300));
    }
    __syncthreads();
    const double piv = L[j][j];
    for (int r = j + 1 + tid; r < b; r += blockDim.x) L[r][j] /= piv;
    __syncthreads();
    for (int e = tid; e < (b - j - 1) * (b - j - 1); e += blockDim.x) {
      const int r = j + 1 + e / (b - j - 1), c = j + 1 + e % (b - j - 1);
      if (c <= r) L[r][c] -= L[r][j] * L[c][j];
    }
    __syncthreads();
  }
  // Li = L^-1 (lower): column by column forward substitution, one thread per column
  for (int c = tid; c < b; c += blockDim.x) {
    for (int r = 0; r < b; ++r) {
      double s = (r == c) ? 1.0 : 0.0;
      for (int q = c; q < r; ++q) s -= L[r][q] * Li[q][c];
      Li[r][c] = (r >= c) ? s / L[r][r] : 0.0;
    }
  }
  __syncthreads();
  // P = Li^T Li
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int r = e / b, c = e % b;
    double s = 0.0;
    const int q0 = r > c ? r : c;
    for (int q = q0; q < b; ++q) s += Li[q][r] * Li[q][c];
    P[r * b + c] = s;
  }
  if (tid == 0 && bad) atomicOr(flag, 1);
}

// Copy a rows x cols block: dst[r*ldd + c] = src[r*lds + c] * scale (zero rows in [z0, z1)).
__global__ void k_copy_block(const double* src, long long lds, double* dst, long long ldd, int rows, int cols,
                             double scale, int z0, int z1) {
  const long long tot = (long long)rows * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e % cols);
    dst[(size_t)r * ldd + c] = (r >= z0 && r < z1) ? 0.0 : scale * src[(size_t)r * lds + c];
  }
}

}  // namespace mvsk
