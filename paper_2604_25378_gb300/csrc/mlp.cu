// Learned warm start of the batched solver: a ReLU multilayer perceptron on
// the tcgen05 GEMM of gemm_tc.cuh (BF16 operands, FP32 accumulation), its
// backward pass, Adam, the request features and the projection of its output
// onto Delta(tau).  The C ABI is declared in include/mvsk_mlp.h.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <vector>

#include "gemm_tc.cuh"
#include "internal.h"
#include "mvsk.h"
#include "mvsk_mlp.h"
#include "vec.cuh"

namespace mvsk {
namespace {

constexpr int kSketch = 32;  // projections per column statistic
constexpr float kB1 = 0.9f, kB2 = 0.999f, kEps = 1e-8f;
constexpr int kLossBlocks = 256;

mvsk_status mfail(mvsk_status st, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return st;
}

#define MCU(x)                                                                                              \
  do {                                                                                                      \
    cudaError_t e_ = (x);                                                                                   \
    if (e_ != cudaSuccess) return mfail(MVSK_ECUDA, "%s: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, \
                                        __LINE__);                                                          \
  } while (0)
#define MTRY(x)                     \
  do {                              \
    const mvsk_status s_ = (x);     \
    if (s_ != MVSK_OK) return s_;   \
  } while (0)

// ----------------------------------------------------------------- epilogue
// Dense layer: z = acc + bias[n]; Z[m*ldz + n] = z (FP32, nullable);
// Abf[m*lda + n] = bf16(relu ? max(z, 0) : z) (nullable).  Each thread holds
// CW consecutive columns of its row m, stored contiguously.
struct EpiDense {
  float* Z;
  long long ldz;
  __nv_bfloat16* Abf;
  long long lda;
  const float* bias;
  int M, N, relu;
  template <int CW>
  __device__ __forceinline__ void operator()(int m, int n0, const float (&v)[CW], int) const {
    if (m >= M) return;
#pragma unroll
    for (int i = 0; i < CW; ++i) {
      const int n = n0 + i;
      if (n < N) {
        const float z = v[i] + (bias != nullptr ? bias[n] : 0.f);
        if (Z != nullptr) Z[(size_t)m * ldz + n] = z;
        if (Abf != nullptr) Abf[(size_t)m * lda + n] = __float2bfloat16(relu ? fmaxf(z, 0.f) : z);
      }
    }
  }
};

// ----------------------------------------------------------------- kernels
__global__ void k_to_bf16(const float* x, __nv_bfloat16* y, size_t cnt) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// He-normal weights: W[o][i] = sqrt(2 / din) * normal(seed, layer, o * din + i).
__global__ void k_init_w(float* W, __nv_bfloat16* Wb, int dout, int din, unsigned long long seed, int layer) {
  const size_t cnt = (size_t)dout * din;
  const double sc = sqrt(2.0 / (double)din);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x) {
    const float w = (float)(sc * probe_value(seed, layer, 0, (int)i));
    W[i] = w;
    Wb[i] = __float2bfloat16(w);
  }
}

// out[c*ldo + r] = in[r*ldi + c] for r < R, c < C; zero for R <= r < Rp (32 x 32 tiles).
__global__ void k_transpose(const __nv_bfloat16* in, int R, int C, long long ldi, __nv_bfloat16* out, long long ldo,
                            int Rp) {
  __shared__ __nv_bfloat16 tile[32][34];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * ldi + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (c < C && r < Rp) out[(size_t)c * ldo + r] = tile[threadIdx.x][k];
  }
}

// dY = 2 (y - t) / (B n) (FP32 and BF16); part[block] = sum of (y - t)^2 over
// the block's elements (FP64, fixed order within the block).
__global__ void __launch_bounds__(256) k_loss_grad(const float* Y, const float* Tt, size_t cnt, float scale,
                                                   float* dY, __nv_bfloat16* dYb, double* part) {
  __shared__ double scr[64];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - Tt[i];
    s += (double)d * (double)d;
    const float g = 2.f * d * scale;
    dY[i] = g;
    dYb[i] = __float2bfloat16(g);
  }
  s = block_sum(s, scr);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_parts(const double* part, int G, double scale, double* out) {
  __shared__ double scr[64];
  double s = 0.0;
  for (int i = threadIdx.x; i < G; i += blockDim.x) s += part[i];
  s = block_sum(s, scr);
  if (threadIdx.x == 0) *out = s * scale;
}

// dZ = bf16(dA o [Z > 0]).
__global__ void k_relu_bwd(const float* dA, const float* Z, __nv_bfloat16* dZ, size_t cnt) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x)
    dZ[i] = __float2bfloat16(Z[i] > 0.f ? dA[i] : 0.f);
}

// db[n] = sum_b dA[b][n] [Z[b][n] > 0] (Z nullable: no mask), FP64 accumulation.
__global__ void k_colsum(const float* dA, const float* Z, int B, int N, float* db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double s = 0.0;
  for (int b = 0; b < B; ++b) {
    const size_t k = (size_t)b * N + n;
    if (Z == nullptr || Z[k] > 0.f) s += (double)dA[k];
  }
  db[n] = (float)s;
}

// Adam on cnt parameters; the BF16 copy (nullable) follows the master weights.
__global__ void k_adam(float* w, float* m, float* v, const float* g, size_t cnt, float lr, float bc1, float bc2,
                       __nv_bfloat16* wb) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = kB1 * m[i] + (1.f - kB1) * gi;
    const float vi = kB2 * v[i] + (1.f - kB2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + kEps);
    w[i] = wi;
    if (wb != nullptr) wb[i] = __float2bfloat16(wi);
  }
}

// st = {mean mu, std mu, mean sigma, std sigma} (population std, two passes).
__global__ void __launch_bounds__(1024) k_stats(const double* mu, const double* sg, int n, double* st) {
  __shared__ double scr[80];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a += mu[i];
    b += sg[i];
  }
  const double2 s1 = block_sum2(a, b, scr);
  const double ma = s1.x / n, mb = s1.y / n;
  a = b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a += (mu[i] - ma) * (mu[i] - ma);
    b += (sg[i] - mb) * (sg[i] - mb);
  }
  const double2 s2 = block_sum2(a, b, scr);
  if (threadIdx.x == 0) {
    st[0] = ma;
    st[1] = sqrt(s2.x / n);
    st[2] = mb;
    st[3] = sqrt(s2.y / n);
  }
}

// sk[r] = P_r . u, u the standardised (mean 0, norm 1) mu (r < kSketch) or
// sigma (otherwise), P_r[i] the probe normal (seed, iteration 0, k = r, i).
__global__ void __launch_bounds__(1024) k_sketch(const double* mu, const double* sg, int n, const double* st,
                                                 unsigned long long seed, double* sk) {
  __shared__ double scr[80];
  const int r = blockIdx.x;
  const double* s = r < kSketch ? mu : sg;
  const double m = r < kSketch ? st[0] : st[2], sd = r < kSketch ? st[1] : st[3];
  double acc = 0.0;
  if (sd > 0.0) {
    const double inv = 1.0 / (sd * sqrt((double)n));
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += probe_value(seed, 0, r, i) * ((s[i] - m) * inv);
  }
  acc = block_sum2(acc, 0.0, scr).x;
  if (threadIdx.x == 0) sk[r] = acc;
}

// X[b][:] = (lambda_b, target feature, flag, sketch, 0 ...).
__global__ void k_feature_rows(const double* lam, const double* tg, int B, const double* st, const double* sk,
                               float* X) {
  const int j = threadIdx.x, b = blockIdx.x;
  if (b >= B || j >= MVSK_MLP_D_IN) return;
  double v = 0.0;
  if (j < 4) {
    v = lam[(size_t)b * 4 + j];
  } else if (j < 6) {
    const double t = tg[b];
    if (isfinite(t)) v = j == 5 ? 1.0 : (st[1] > 0.0 ? (t - st[0]) / st[1] : 0.0);
  } else if (j < 6 + 2 * kSketch) {
    v = sk[j - 6];
  }
  X[(size_t)b * MVSK_MLP_D_IN + j] = (float)v;
}

// W0[b] = Pi_Delta(tau)(Y[b] * scale): one CTA per row (Michelot threshold).
__global__ void __launch_bounds__(1024) k_project_rows(const float* Y, int ldy, int n, double scale, double tau,
                                                       double* W0) {
  __shared__ double scr[80];
  double* w = W0 + (size_t)blockIdx.x * n;
  const float* y = Y + (size_t)blockIdx.x * ldy;
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = (double)y[i] * scale;
  __syncthreads();
  const double th = slice_theta(w, nullptr, 0.0, n, tau, scr, w);  // w now holds y*scale - tau
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = tau + fmax(w[i] - th, 0.0);
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// K-major BF16 operand (rows x K, row stride ld elements) for a 64 x box_rows TMA box.
mvsk_status tmap(CUtensorMap* tm, const __nv_bfloat16* base, long long K, long long rows, long long ld,
                 unsigned box_rows) {
  auto enc = encoder();
  if (enc == nullptr) return mfail(MVSK_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || ((ld * 2) & 15) != 0)
    return mfail(MVSK_EINVAL, "GEMM operand base or row stride not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTcBK, box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return mfail(MVSK_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return MVSK_OK;
}

constexpr int kGBN = 64;  // N tile of the network's GEMMs

}  // namespace
}  // namespace mvsk

using namespace mvsk;

struct mvsk_mlp {
  int L = 0, maxb = 0, maxbp = 0, maxdim = 0;
  std::vector<int> dims;  // dims[0] = d_in ... dims[L] = d_out
  std::vector<float*> W, b, mW, vW, mb, vb, gW, gb, Z;
  std::vector<__nv_bfloat16*> Wb, Wt, Ab;
  float* dA = nullptr;
  float* dY = nullptr;
  __nv_bfloat16* dZb = nullptr;
  __nv_bfloat16* dZt = nullptr;
  __nv_bfloat16* At = nullptr;
  double* part = nullptr;
  double* lossd = nullptr;
  double* feat = nullptr;  // stats (4) + sketch (64)
  int* err = nullptr;
  long long step = 0;
  std::vector<void*> allocs;
  cudaStream_t stream = nullptr;
};

namespace {

template <typename T>
mvsk_status alloc(mvsk_mlp* p, T** ptr, size_t cnt) {
  void* q = nullptr;
  if (cudaMalloc(&q, cnt * sizeof(T) + 16) != cudaSuccess) return mfail(MVSK_ENOMEM, "device allocation failed");
  p->allocs.push_back(q);
  if (cudaMemset(q, 0, cnt * sizeof(T) + 16) != cudaSuccess) return mfail(MVSK_ECUDA, "cudaMemset failed");
  *ptr = static_cast<T*>(q);
  return MVSK_OK;
}

unsigned blocks_for(size_t cnt) {
  const size_t b = (cnt + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// C[m, n] = sum_k A[m, k] B[n, k] for A (M x K, ld lda), B (N x K, ld ldb) into epi.
mvsk_status gemm(mvsk_mlp* p, const __nv_bfloat16* A, int M, long long lda, const __nv_bfloat16* Bm, int N,
                 long long ldb, int K, const EpiDense& epi) {
  CUtensorMap ta, tb;
  MTRY(tmap(&ta, A, K, M, lda, kTcBM));
  MTRY(tmap(&tb, Bm, K, N, ldb, kGBN));
  const int nk = (K + kTcBK - 1) / kTcBK;
  const dim3 grid((unsigned)((N + kGBN - 1) / kGBN), (unsigned)((M + kTcBM - 1) / kTcBM), 1);
  k_gemm_tc<kGBN, 4, EpiDense, 1><<<grid, 128, tc_smem_bytes<kGBN, 4, 1>(), p->stream>>>(ta, tb, M, N, K, nk, epi,
                                                                                         p->err, nullptr, nullptr);
  MCU(cudaGetLastError());
  return MVSK_OK;
}

mvsk_status check_err(mvsk_mlp* p) {
  int e = 0;
  MCU(cudaMemcpyAsync(&e, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  MCU(cudaStreamSynchronize(p->stream));
  if (e != 0) return mfail(MVSK_ECUDA, "a bounded in-kernel wait ran out (error word %d)", e);
  return MVSK_OK;
}

// Forward pass of B rows of X (FP32, B x d_in): Ab[0] = bf16(X), Z[l], Ab[l + 1].
mvsk_status forward(mvsk_mlp* p, const float* X, int B) {
  const size_t cin = (size_t)B * p->dims[0];
  k_to_bf16<<<blocks_for(cin), 256, 0, p->stream>>>(X, p->Ab[0], cin);
  MCU(cudaGetLastError());
  for (int l = 0; l < p->L; ++l) {
    const bool hidden = l + 1 < p->L;
    EpiDense e{p->Z[l], p->dims[l + 1], hidden ? p->Ab[l + 1] : nullptr, p->dims[l + 1], p->b[l], B, p->dims[l + 1],
               hidden ? 1 : 0};
    MTRY(gemm(p, p->Ab[l], B, p->dims[l], p->Wb[l], p->dims[l + 1], p->dims[l], p->dims[l], e));
  }
  return MVSK_OK;
}

mvsk_status check_batch(mvsk_mlp* p, int B) {
  if (p == nullptr) return mfail(MVSK_EINVAL, "null network");
  if (B < 1 || B > p->maxb) return mfail(MVSK_EINVAL, "batch %d outside [1, %d]", B, p->maxb);
  return MVSK_OK;
}

}  // namespace

extern "C" {

mvsk_status mvsk_mlp_create(int32_t d_in, int32_t d_hidden, int32_t n_hidden, int32_t d_out, int32_t max_batch,
                            uint64_t seed, mvsk_mlp** out) {
  if (out == nullptr) return mfail(MVSK_EINVAL, "null output pointer");
  *out = nullptr;
  if (d_in < 8 || d_hidden < 8 || d_out < 8 || n_hidden < 1 || max_batch < 8 || d_in % 8 || d_hidden % 8 ||
      d_out % 8 || max_batch % 8)
    return mfail(MVSK_EINVAL, "dimensions must be multiples of 8 (>= 8) and n_hidden >= 1");
  static bool attr = false;
  if (!attr) {
    MCU(cudaFuncSetAttribute(k_gemm_tc<kGBN, 4, EpiDense, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_smem_bytes<kGBN, 4, 1>()));
    attr = true;
  }
  mvsk_mlp* p = new mvsk_mlp();
  p->L = n_hidden + 1;
  p->dims.push_back(d_in);
  for (int l = 0; l < n_hidden; ++l) p->dims.push_back(d_hidden);
  p->dims.push_back(d_out);
  p->maxb = max_batch;
  p->maxbp = max_batch;
  for (int d : p->dims) p->maxdim = d > p->maxdim ? d : p->maxdim;
  auto fail_free = [&](mvsk_status st) {
    mvsk_mlp_destroy(p);
    return st;
  };
  const int L = p->L;
  p->W.resize(L); p->b.resize(L); p->mW.resize(L); p->vW.resize(L); p->mb.resize(L); p->vb.resize(L);
  p->gW.resize(L); p->gb.resize(L); p->Z.resize(L); p->Wb.resize(L); p->Wt.resize(L); p->Ab.resize(L);
  mvsk_status st = MVSK_OK;
  for (int l = 0; l < L && st == MVSK_OK; ++l) {
    const size_t nw = (size_t)p->dims[l + 1] * p->dims[l], nb = (size_t)p->dims[l + 1];
    if ((st = alloc(p, &p->W[l], nw)) || (st = alloc(p, &p->mW[l], nw)) || (st = alloc(p, &p->vW[l], nw)) ||
        (st = alloc(p, &p->gW[l], nw)) || (st = alloc(p, &p->Wb[l], nw)) || (st = alloc(p, &p->Wt[l], nw)) ||
        (st = alloc(p, &p->b[l], nb)) || (st = alloc(p, &p->mb[l], nb)) || (st = alloc(p, &p->vb[l], nb)) ||
        (st = alloc(p, &p->gb[l], nb)) || (st = alloc(p, &p->Z[l], (size_t)max_batch * nb)) ||
        (st = alloc(p, &p->Ab[l], (size_t)max_batch * p->dims[l])))
      break;
  }
  if (st == MVSK_OK) {
    const size_t big = (size_t)max_batch * p->maxdim;
    if ((st = alloc(p, &p->dA, big)) || (st = alloc(p, &p->dY, (size_t)max_batch * d_out)) ||
        (st = alloc(p, &p->dZb, big)) || (st = alloc(p, &p->dZt, big)) || (st = alloc(p, &p->At, big)) ||
        (st = alloc(p, &p->part, (size_t)kLossBlocks)) || (st = alloc(p, &p->lossd, (size_t)1)) ||
        (st = alloc(p, &p->feat, (size_t)4 + 2 * kSketch)) || (st = alloc(p, &p->err, (size_t)1))) {
    }
  }
  if (st != MVSK_OK) return fail_free(st);
  for (int l = 0; l < L; ++l) {
    const int dout = p->dims[l + 1], din = p->dims[l];
    k_init_w<<<blocks_for((size_t)dout * din), 256, 0, p->stream>>>(p->W[l], p->Wb[l], dout, din, seed, l);
    k_transpose<<<dim3((din + 31) / 32, (dout + 31) / 32), dim3(32, 8), 0, p->stream>>>(p->Wb[l], dout, din, din,
                                                                                        p->Wt[l], dout, dout);
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(p->stream) != cudaSuccess)
    return fail_free(mfail(MVSK_ECUDA, "network initialisation failed"));
  *out = p;
  return MVSK_OK;
}

mvsk_status mvsk_mlp_destroy(mvsk_mlp* p) {
  if (p == nullptr) return MVSK_OK;
  cudaStreamSynchronize(p->stream);
  for (void* q : p->allocs) cudaFree(q);
  delete p;
  return MVSK_OK;
}

mvsk_status mvsk_mlp_forward(mvsk_mlp* p, const float* X, int32_t B, float* Y) {
  MTRY(check_batch(p, B));
  MTRY(forward(p, X, B));
  MCU(cudaMemcpyAsync(Y, p->Z[p->L - 1], sizeof(float) * (size_t)B * p->dims[p->L], cudaMemcpyDefault, p->stream));
  return check_err(p);
}

mvsk_status mvsk_mlp_train_step(mvsk_mlp* p, const float* X, const float* Yt, int32_t B, float lr, double* loss) {
  MTRY(check_batch(p, B));
  const int L = p->L, dout = p->dims[L];
  const int Bp = (B + 7) / 8 * 8;
  MTRY(forward(p, X, B));
  const size_t cnt = (size_t)B * dout;
  k_loss_grad<<<kLossBlocks, 256, 0, p->stream>>>(p->Z[L - 1], Yt, cnt, 1.f / (float)cnt, p->dY, p->dZb, p->part);
  k_sum_parts<<<1, 256, 0, p->stream>>>(p->part, kLossBlocks, 1.0 / (double)cnt, p->lossd);
  MCU(cudaGetLastError());
  for (int l = L - 1; l >= 0; --l) {
    const int din = p->dims[l], dl = p->dims[l + 1];
    // bias gradient from the FP32 error: dY at the output, dA o [Z > 0] below
    k_colsum<<<(dl + 255) / 256, 256, 0, p->stream>>>(l == L - 1 ? p->dY : p->dA, l == L - 1 ? nullptr : p->Z[l], B,
                                                       dl, p->gb[l]);
    // dW = dZ^T A_{l}: both operands K-major in the batch (transposed, zero-padded to Bp)
    k_transpose<<<dim3((dl + 31) / 32, (Bp + 31) / 32), dim3(32, 8), 0, p->stream>>>(p->dZb, B, dl, dl, p->dZt, Bp,
                                                                                      Bp);
    k_transpose<<<dim3((din + 31) / 32, (Bp + 31) / 32), dim3(32, 8), 0, p->stream>>>(p->Ab[l], B, din, din, p->At,
                                                                                       Bp, Bp);
    MCU(cudaGetLastError());
    EpiDense eg{p->gW[l], din, nullptr, 0, nullptr, dl, din, 0};
    MTRY(gemm(p, p->dZt, dl, Bp, p->At, din, Bp, Bp, eg));
    if (l > 0) {
      // dA_{l-1} = dZ W (W^T stored K-major in the layer's output), then dZ_{l-1}
      EpiDense ea{p->dA, din, nullptr, 0, nullptr, B, din, 0};
      MTRY(gemm(p, p->dZb, B, dl, p->Wt[l], din, dl, dl, ea));
      const size_t c2 = (size_t)B * din;
      k_relu_bwd<<<blocks_for(c2), 256, 0, p->stream>>>(p->dA, p->Z[l - 1], p->dZb, c2);
      MCU(cudaGetLastError());
    }
  }
  p->step += 1;
  const float bc1 = 1.f - powf(kB1, (float)p->step), bc2 = 1.f - powf(kB2, (float)p->step);
  for (int l = 0; l < L; ++l) {
    const int din = p->dims[l], dl = p->dims[l + 1];
    const size_t nw = (size_t)dl * din;
    k_adam<<<blocks_for(nw), 256, 0, p->stream>>>(p->W[l], p->mW[l], p->vW[l], p->gW[l], nw, lr, bc1, bc2, p->Wb[l]);
    k_adam<<<blocks_for(dl), 256, 0, p->stream>>>(p->b[l], p->mb[l], p->vb[l], p->gb[l], (size_t)dl, lr, bc1, bc2,
                                                  nullptr);
    k_transpose<<<dim3((din + 31) / 32, (dl + 31) / 32), dim3(32, 8), 0, p->stream>>>(p->Wb[l], dl, din, din,
                                                                                      p->Wt[l], dl, dl);
  }
  MCU(cudaGetLastError());
  if (loss != nullptr) MCU(cudaMemcpyAsync(loss, p->lossd, sizeof(double), cudaMemcpyDefault, p->stream));
  return check_err(p);
}

mvsk_status mvsk_mlp_access(mvsk_mlp* p, int32_t layer, int32_t what, float* W, float* b) {
  if (p == nullptr || layer < 0 || layer >= p->L || what < 0 || what > 2)
    return mfail(MVSK_EINVAL, "bad layer %d or access kind %d", (int)layer, (int)what);
  const int din = p->dims[layer], dl = p->dims[layer + 1];
  const size_t nw = (size_t)dl * din;
  if (what == 1) {
    if (W != nullptr) {
      MCU(cudaMemcpyAsync(p->W[layer], W, sizeof(float) * nw, cudaMemcpyDefault, p->stream));
      k_to_bf16<<<blocks_for(nw), 256, 0, p->stream>>>(p->W[layer], p->Wb[layer], nw);
      k_transpose<<<dim3((din + 31) / 32, (dl + 31) / 32), dim3(32, 8), 0, p->stream>>>(p->Wb[layer], dl, din, din,
                                                                                        p->Wt[layer], dl, dl);
      MCU(cudaGetLastError());
    }
    if (b != nullptr) MCU(cudaMemcpyAsync(p->b[layer], b, sizeof(float) * dl, cudaMemcpyDefault, p->stream));
  } else {
    const float* sw = what == 0 ? p->W[layer] : p->gW[layer];
    const float* sb = what == 0 ? p->b[layer] : p->gb[layer];
    if (W != nullptr) MCU(cudaMemcpyAsync(W, sw, sizeof(float) * nw, cudaMemcpyDefault, p->stream));
    if (b != nullptr) MCU(cudaMemcpyAsync(b, sb, sizeof(float) * dl, cudaMemcpyDefault, p->stream));
  }
  MCU(cudaStreamSynchronize(p->stream));
  return MVSK_OK;
}

mvsk_status mvsk_mlp_features(const double* mu, const double* sigma, int64_t n, int32_t B, const double* lambda,
                              const double* target, uint64_t seed, float* X) {
  if (n < 2 || n > 0x7fffffff || B < 1 || mu == nullptr || sigma == nullptr || lambda == nullptr ||
      target == nullptr || X == nullptr)
    return mfail(MVSK_EINVAL, "bad feature arguments (n %lld, B %d)", (long long)n, (int)B);
  double* buf = nullptr;
  MCU(cudaMalloc(&buf, sizeof(double) * (4 + 2 * kSketch)));
  k_stats<<<1, 1024>>>(mu, sigma, (int)n, buf);
  k_sketch<<<2 * kSketch, 1024>>>(mu, sigma, (int)n, buf, (unsigned long long)seed, buf + 4);
  k_feature_rows<<<B, MVSK_MLP_D_IN>>>(lambda, target, B, buf, buf + 4, X);
  const cudaError_t e = cudaGetLastError();
  const cudaError_t s = cudaDeviceSynchronize();
  cudaFree(buf);
  if (e != cudaSuccess || s != cudaSuccess) return mfail(MVSK_ECUDA, "feature kernels failed");
  return MVSK_OK;
}

mvsk_status mvsk_mlp_warm_start(mvsk_mlp* p, const float* X, int32_t B, int64_t n, double tau, double* W0) {
  MTRY(check_batch(p, B));
  if (n != p->dims[p->L]) return mfail(MVSK_EINVAL, "n = %lld differs from the output width %d", (long long)n,
                                       p->dims[p->L]);
  if (!(tau >= 0.0) || tau * (double)n >= 1.0) return mfail(MVSK_EINVAL, "tau outside [0, 1/n)");
  MTRY(forward(p, X, B));
  k_project_rows<<<B, 1024, 0, p->stream>>>(p->Z[p->L - 1], p->dims[p->L], (int)n, 1.0 / (double)n, tau, W0);
  MCU(cudaGetLastError());
  return check_err(p);
}

}  // extern "C"
