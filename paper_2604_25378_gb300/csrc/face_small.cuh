// Direction block of a lockstep batch when every working face is small
// (included into batch_impl.cuh).
//
// After the first steps of a solve the working face F of an instance holds a
// few dozen coordinates.  The PCG configuration then needs the tangent
// Hessian only on F: G_F = T^-1 A_F^T Diag(psi''(z)) A_F (Prop. 2) is an
// m x m matrix (m = |F| <= kMF), formed once per iteration from the columns of
// A in F, after which every Hessian-vector product of both PCG rounds is
// G_F p (Eq. operator-hvp restricted to F, the same numbers as
// T^-1 A^T (psi'' o A p) for p supported on F) and a whole PCG round runs in
// one CTA per (instance, column) with G_F in shared memory.  The Hutchinson
// correction a = T^-1 A_F^T (psi''' o rhat), rhat = K^-1 sum_k (A_F X_k) o
// (A_F p_k) (Eq. operator-third), takes one more pass over A_F.  The columns
// of A come from the union gather of the face-restricted products (BF16, the
// precision of the other direction products).  G_F and the correction's two
// contractions run on the tensor cores (BF16 data, the weighted or iterate
// operand carried in two BF16 parts, FP32 accumulation); the PCG recurrences
// and the set-ups are FP32 with FP64 block sums.  Two launch shapes: NM =
// kMFt while every face has at most kMFt coordinates, NM = kMF otherwise.
#pragma once

constexpr int kMF = 320;       // largest face handled here (one coordinate per thread of a PCG CTA)
constexpr int kMFt = 128;      // faces up to this size take the narrow instantiation (NM = kMFt)

// Face list of instance blockIdx.y: fl[k] = i for the coordinates of its
// working face (maskF = 1) in increasing order, si[SI_FCNT] = their count.
// One CTA of 1024 threads per instance.
__global__ void __launch_bounds__(1024) k_face_list(Inst base, int* fl_base) {
  const Inst s = inst_at(base, blockIdx.y);
  if (s.si[SI_DONE] != 0 || s.si[SI_SKIPDIR] != 0) return;
  int* fl = fl_base + (size_t)blockIdx.y * s.vs;
  __shared__ int wsum[32];
  const int n = s.n, per = (n + 1023) / 1024, i0 = threadIdx.x * per;
  int cnt = 0;
  for (int i = i0; i < i0 + per && i < n; ++i) cnt += s.maskF[i] != 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int v = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  int p = v - cnt + (warp > 0 ? wsum[warp - 1] : 0);
  for (int i = i0; i < i0 + per && i < n; ++i)
    if (s.maskF[i] != 0.0) fl[p++] = i;
  if (threadIdx.x == 1023) s.si[SI_FCNT] = p;
}

// info[2] = 2 when every instance that needs a direction this iteration has a
// face of at most kMFt coordinates (the narrow small-face block runs), else 1
// when every such face has at most kMF (the wide one), else 0 (also when
// small = 0).  wide != 0 takes the wide block for every small face.  With
// has_cond the same value selects the body of the iteration graph's switch
// node (handle cond).
__global__ void k_small_mode(Inst base, int B, int small, int wide, int* info, cudaGraphConditionalHandle cond,
                             int has_cond) {
  int big = 0, mid = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int* si = base.si + (size_t)b * kSI;
    if (si[SI_DONE] == 0 && si[SI_SKIPDIR] == 0) {
      big |= si[SI_FCNT] > kMF;
      mid |= si[SI_FCNT] > kMFt;
    }
  }
  big = __syncthreads_or(big);
  mid = __syncthreads_or(mid | wide);
  if (threadIdx.x == 0) {
    const int f = (big || !small) ? 0 : (mid ? 1 : 2);
    info[2] = f;
    if (has_cond) cudaGraphSetConditional(cond, (unsigned)f);
  }
}

// Face Grams on the tensor cores.  CTA (x, b, t) accumulates over the 64-row
// blocks [x nkb / S, (x + 1) nkb / S) of instance b (S = gridDim.x) the rows
// 128 t .. 128 t + 127 of D = P Q^T with P[k][t] = a_tk (face coordinate k,
// a row of the gathered A^T: AUT row upos[fl[k]], ldt BF16 apart, contiguous
// in t) and Q[l][t] = psi2(z_t) a_tl split into BF16 parts Q = Qhi + Qlo (Qhi
// the rounding of the FP32 product, Qlo that of the rest; together ~16 bits),
// so that D = P Qhi^T + P Qlo^T is sum_t psi2(z_t) a_tk a_tl to about the
// precision of FP32 products of the BF16 data (FP32 accumulation in TMEM):
// M = 128 (this CTA's tile of the face), N = m rounded up to 16 (<= kMF, in
// pieces of at most 256), K = 64 rows of A per stage.  The 256 threads stage
// the operands (16-byte loads along t, as 128-byte swizzled K-major rows, the
// layout the MMA descriptors read) into one of two stages while the MMAs of
// the other run, the loads of the next block in flight; thread 0 issues the
// MMAs.  Out: element (k, l), k <= l < m, k in the tile, of slab (b, x) at
// k mp8 + l (mp8 = m rounded up to 8): the partial layout k_face_gram_sum
// adds.  Dynamic shared memory kGramTcSmem; waits are bounded (err |=
// kErrWaitTimeout on expiry).
constexpr int kGTBytesA = 128 * 128;  // one M tile of 128 rows x 64 BF16
// Shapes of the instantiation for faces of at most NM coordinates.
template <int NM>
struct GramTc {
  static constexpr int kBytesB = NM * 128;              // up to NM rows x 64 BF16 (one of Qhi, Qlo)
  static constexpr int kChunks = ((NM + 127) / 128) * 128 * 8 / 256;  // 16-byte chunks per thread and block
  static constexpr size_t kSmem = 1024 + (size_t)2 * (kGTBytesA + 2 * kBytesB) + 256;
  static constexpr int kTmemCols = NM <= 128 ? 128 : (NM <= 256 ? 256 : 512);
  static constexpr int kSplit = NM <= kMFt ? 8 : 2;     // shares of the rows of A per instance
  static constexpr int kDepth = NM <= kMFt ? 2 : 1;     // 64-row blocks loaded ahead
  static constexpr int kMinBlocks = NM <= kMFt ? 2 : 1;  // resident CTAs per SM (shared memory)
  static_assert(NM % 16 == 0 && NM <= 512, "the N extent of the face Gram MMA");
};
constexpr int kGramSplit = GramTc<kMF>::kSplit;
static_assert(GramTc<kMFt>::kSplit * kMFt * kMFt <= kGramSplit * kMF * kMF, "partial Grams of the narrow block");

// Asynchronous global -> shared copies (cp.async): 16 bytes (zero-filled
// when !full), 4 bytes; groups committed and waited for by each thread.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool full) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(full ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ int sw128_off(int r, int j) {
  return ((r >> 3) << 10) + ((r & 7) << 7) + (((j ^ r) & 7) << 4);
}

// 8 BF16 values (a uint4) times h[0..7] in FP32, split into BF16 parts:
// *hi the rounding of each product, *lo the rounding of its remainder.
__device__ __forceinline__ void bf16x8_scale2(uint4 v, const float* h, uint4* hi, uint4* lo) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint32_t a[4], c[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float p0 = __uint_as_float(w[q] << 16) * h[2 * q], p1 = __uint_as_float(w[q] & 0xFFFF0000u) * h[2 * q + 1];
    const __nv_bfloat162 r2 = __floats2bfloat162_rn(p0, p1);
    const float2 rf = __bfloat1622float2(r2);
    const __nv_bfloat162 e2 = __floats2bfloat162_rn(p0 - rf.x, p1 - rf.y);
    a[q] = *reinterpret_cast<const uint32_t*>(&r2);
    c[q] = *reinterpret_cast<const uint32_t*>(&e2);
  }
  *hi = make_uint4(a[0], a[1], a[2], a[3]);
  *lo = make_uint4(c[0], c[1], c[2], c[3]);
}

template <int NM>
__global__ void __launch_bounds__(256, GramTc<NM>::kMinBlocks)
    k_face_gram_tc(Inst base, const int* fl_base, const __nv_bfloat16* AUT, long long ldt, const int* upos, float* gp,
                   int* err) {
  using G = GramTc<NM>;
  constexpr int kGTBytesB = G::kBytesB, kGTChunks = G::kChunks;
  const int b = blockIdx.y, mt = blockIdx.z;
  const Inst s = inst_at(base, b);
  if (s.si[SI_DONE] != 0 || s.si[SI_SKIPDIR] != 0) return;
  const int m = s.si[SI_FCNT];
  if (m > NM || m <= 0 || mt * 128 >= m) return;
  const int n16 = (m + 15) & ~15, mp8 = (m + 7) & ~7;
  const int rows = n16 > mt * 128 + 128 ? n16 : mt * 128 + 128;  // rows staged: Q's and this tile's
  const long long T = s.T;
  const int nkb = (int)((T + 63) / 64);
  const int kb0 = (int)((long long)blockIdx.x * nkb / gridDim.x);
  const int kb1 = (int)((long long)(blockIdx.x + 1) * nkb / gridDim.x);
  if (kb0 >= kb1) return;  // uniform over the CTA, before any barrier or TMEM use
  extern __shared__ unsigned char gsm_raw[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = sm;
  unsigned char* sB = sm + 2 * kGTBytesA;  // per stage: Qhi, then Qlo
  uint64_t* mdone = reinterpret_cast<uint64_t*>(sB + 4 * kGTBytesB);  // [2]: the MMAs of a stage completed
  uint64_t* fin = mdone + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
  __shared__ float h[2 * 64];  // weights of the rows of the block in each stage
  __shared__ int roww[kGTChunks * 32];
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int* fl = fl_base + (size_t)b * s.vs;
  for (int r = tid; r < kGTChunks * 32; r += 256) roww[r] = r < m ? upos[fl[r]] : -1;
  if (tid == 0) {
    mbar_init(&mdone[0], 1);
    mbar_init(&mdone[1], 1);
    mbar_init(fin, 1);
    fence_barrier_init();
    s_abort = 0;
  }
  if (warp == 0) tmem_alloc(tslot, G::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const float c2 = (float)s.sd[SD_C2], c3 = (float)s.sd[SD_C3], c4 = (float)s.sd[SD_C4];
  // G is symmetric and only its upper triangle (l >= k) is kept: the tile of
  // rows nbase .. nbase + 127 needs the columns l >= nbase only (Q rows
  // nbase .. n16, N = n16 - nbase in pieces of at most 256)
  const int nbase = mt * 128, ntot = n16 - nbase, cbase = nbase * 8;
  const int nn0 = ntot < 256 ? ntot : 256, nn1 = ntot - nn0;
  const uint32_t idesc0 = idesc_bf16_f32(kTcBM, nn0), idesc1 = idesc_bf16_f32(kTcBM, nn1 > 0 ? nn1 : 16);
  // Thread tid takes the 16-byte chunks tid + 256 q (row c / 8, chunk c % 8)
  // of a 64-row block, and threads < 64 the weight of row tid.  The loads of
  // block i + 1 are issued at the top of iteration i (registers vn, zn), so
  // that their latency passes while the MMAs of block i - 1 and the staging
  // of block i run.
  // block i + 1 in (vn, zn); with G::kDepth = 2 also block i + 2 in (vn2, zn2)
  uint4 vn[kGTChunks], vn2[kGTChunks];
  double zn = 0.0, zn2 = 0.0;
  auto fetch_into = [&](int kb, uint4 (&dst)[kGTChunks], double& zd) {
    const long long t0 = (long long)kb * 64;
#pragma unroll
    for (int q = 0; q < kGTChunks; ++q) {
      const int c = cbase + tid + 256 * q, r = c >> 3, j = c & 7;
      const long long t = t0 + 8 * j;
      dst[q] = make_uint4(0u, 0u, 0u, 0u);
      if (r < m && t < ldt) dst[q] = __ldg(reinterpret_cast<const uint4*>(AUT + (size_t)roww[r] * ldt + t));
    }
    if (tid < 64 && t0 + tid < T) zd = s.z[t0 + tid];
  };
  auto fetch = [&](int kb) { fetch_into(kb, vn, zn); };
  auto weight = [&](double z64, long long t) {
    const float z = (float)z64;
    return t < T ? 2.f * c2 - z * (6.f * c3 - 12.f * c4 * z) : 0.f;
  };
  fetch(kb0);
  if (G::kDepth == 2 && kb0 + 1 < kb1) fetch_into(kb0 + 1, vn2, zn2);
  if (tid < 64) h[tid] = weight(zn, (long long)kb0 * 64 + tid);
  int i = 0;
  for (int kb = kb0; kb < kb1; ++kb, ++i) {
    const int st = i & 1;
    uint4 v[kGTChunks];
#pragma unroll
    for (int q = 0; q < kGTChunks; ++q) v[q] = vn[q];
    if (G::kDepth == 2) {  // (vn, zn) <- block kb + 1, then block kb + 2 in flight
#pragma unroll
      for (int q = 0; q < kGTChunks; ++q) vn[q] = vn2[q];
      zn = zn2;
      if (kb + 2 < kb1) fetch_into(kb + 2, vn2, zn2);
    } else if (kb + 1 < kb1) {
      fetch(kb + 1);
    }
    if (i >= 2 && !mbar_wait_bounded(&mdone[st], (uint32_t)(((i - 2) >> 1) & 1))) {
      atomicOr(err, kErrWaitTimeout);
      s_abort = 1;
    }
    __syncthreads();  // stage st is free; h[st] holds the weights of this block
    if (s_abort) break;
    unsigned char* pa = sA + (size_t)st * kGTBytesA;
    unsigned char* pb = sB + (size_t)st * 2 * kGTBytesB;
    const float* hb = h + 64 * st;
#pragma unroll
    for (int q = 0; q < kGTChunks; ++q) {
      const int c = cbase + tid + 256 * q, r = c >> 3, j = c & 7;
      if (r >= rows) break;
      if (r < nbase + 128) *reinterpret_cast<uint4*>(pa + sw128_off(r - nbase, j)) = v[q];
      if (r < n16) {
        uint4 qh, ql;
        bf16x8_scale2(v[q], hb + 8 * j, &qh, &ql);
        const int off = sw128_off(r, j);
        *reinterpret_cast<uint4*>(pb + off) = qh;
        *reinterpret_cast<uint4*>(pb + kGTBytesB + off) = ql;
      }
    }
    if (tid < 64 && kb + 1 < kb1) h[64 * (st ^ 1) + tid] = weight(zn, (long long)(kb + 1) * 64 + tid);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint64_t da = umma_desc_sw128(pa);
      const uint64_t dbh = umma_desc_sw128(pb + nbase * 128), dbl = umma_desc_sw128(pb + kGTBytesB + nbase * 128);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        umma_bf16(tmem, da + (uint64_t)(2 * kk), dbh + (uint64_t)(2 * kk), idesc0, acc);
        umma_bf16(tmem, da + (uint64_t)(2 * kk), dbl + (uint64_t)(2 * kk), idesc0, 1u);
        if (nn1 > 0) {  // N rows 256.. of Q: descriptor start 256 rows (32 KB) further
          umma_bf16(tmem + 256u, da + (uint64_t)(2 * kk), dbh + (uint64_t)(256 * 8 + 2 * kk), idesc1, acc);
          umma_bf16(tmem + 256u, da + (uint64_t)(2 * kk), dbl + (uint64_t)(256 * 8 + 2 * kk), idesc1, 1u);
        }
      }
      umma_commit(&mdone[st]);
    }
  }
  if (tid == 0) umma_commit(fin);  // arrives once every MMA issued above has completed
  const bool ok = mbar_wait_bounded(fin, 0);
  if (!ok && tid == 0) atomicOr(err, kErrWaitTimeout);
  tc_fence_after();
  if (ok && !s_abort) {
    // warps w and w + 4 read lane quarter w % 4: the first and second half of the columns
    const int q = warp & 3, half = ((ntot / 2) + 15) & ~15;
    const int k = nbase + q * 32 + lane;
    const int ca = warp < 4 ? 0 : half, cb = warp < 4 ? half : ntot;
    float* out = gp + ((size_t)b * gridDim.x + blockIdx.x) * NM * NM;
    for (int c0 = ca; c0 < cb; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
      if (k < m)
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int l = nbase + c0 + jj;
          if (l >= k && l < m) out[(size_t)k * mp8 + l] = v[jj];
        }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, G::kTmemCols);
}

// Face Gram of instance blockIdx.y from the chunk partials (added in chunk
// order): entries e = k mp + l of the upper triangle handled by CTA
// blockIdx.x (grid-stride), G[k][l] = G[l][k] = T^-1 sum, into
// gram[b * NM * NM] (row stride NM).
template <int NM>
__global__ void __launch_bounds__(256) k_face_gram_sum(Inst base, const float* gp, int nchunk, float* gram) {
  const int b = blockIdx.y;
  const Inst s = inst_at(base, b);
  if (s.si[SI_DONE] != 0 || s.si[SI_SKIPDIR] != 0) return;
  const int m = s.si[SI_FCNT];
  if (m > NM) return;
  const int mp = 8 * ((m + 7) / 8);
  float* Gm = gram + (size_t)b * NM * NM;
  const float invT = (float)s.sd[SD_INVT];
  const float* src0 = gp + (size_t)b * nchunk * NM * NM;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int k = e / m, l = e - k * m;
    if (k > l) continue;
    const float* src = src0 + (size_t)k * mp + l;
    float v = 0.f;
    for (int c = 0; c < nchunk; ++c) v += src[(size_t)c * NM * NM];
    v *= invT;
    Gm[(size_t)k * NM + l] = v;
    Gm[(size_t)l * NM + k] = v;
  }
}

// Sums of six floats over a CTA of NM threads (NM / 32 warps), added in
// warp order so that every thread holds the same totals.
template <int NM>
__device__ __forceinline__ void cta_sum6(float (&v)[6], float (*scr)[6]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 6; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 6; ++q) scr[warp][q] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < NM / 32; ++w) t += scr[w][q];
    v[q] = t;
  }
}

// Sums of Q doubles over a CTA of NM threads, added in warp order so that
// every thread holds the same totals.
template <int NM, int Q>
__device__ __forceinline__ void cta_sumd(double (&v)[Q], double (*scr)[Q]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < Q; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < Q; ++q) scr[warp][q] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NM / 32; ++w) t += scr[w][q];
    v[q] = t;
  }
  __syncthreads();  // scr is free again
}

// d = X_h - (||gbar|| / m) X_a - nuhat on F, re-centred on F (1^T d = 0 to
// rounding), zero elsewhere: k_assemble restricted to F (X_h, X_a and nuhat
// vanish off F), with xa this thread's coordinate of X_a.
template <int NM>
__device__ __forceinline__ void face_assemble(Inst& s, const int* fl_base, int ca, float xa) {
  __shared__ double ascr[NM / 32][1];
  const int m = s.si[SI_FCNT], k = threadIdx.x;
  const bool on = k < m;
  const int* fl = fl_base + (size_t)blockIdx.y * s.vs;
  const int i = on ? fl[k] : 0;
  const double mdim = (double)s.si[SI_M], coef = s.sd[SD_GN] / mdim;
  const double v = on ? (double)kcol<float>(s.X, 0, s.ld)[i] - coef * (double)xa - s.nuhat[i] : 0.0;
  for (int j = threadIdx.x; j < s.ld; j += blockDim.x) s.d[j] = 0.0;
  double sv[1] = {v};
  cta_sumd<NM, 1>(sv, ascr);  // its barriers also order the zeros before the face values
  if (on) s.d[i] = v - sv[0] / mdim;
}

// Start of PCG column c on the face (one coordinate k < m per thread, i =
// fl[k]): right-hand side B = P_V v (v = G nuhat for c = 0, the probe
// otherwise; P_V v = v - mean_F v - (nuhat^T v) nuhat on F), X = 0, R = B,
// P = Z = P_V(B / dg), rz = R^T Z, rhsn = ||B||, active flag, step count 0:
// k_pcg_setup_cols / pcg_init_col restricted to F, where every vector of the
// round lives.  Returns B.
template <int NM>
__device__ __forceinline__ float face_col_start(Inst& s, int c, bool on, int i, float v, float nh, float dg,
                                                double m, double (*scr)[2]) {
  double ab[2] = {on ? (double)v : 0.0, on ? (double)(nh * v) : 0.0};
  cta_sumd<NM, 2>(ab, scr);
  const float mean = (float)(ab[0] / m), ny = (float)ab[1];
  const float Bk = on ? (v - mean) - ny * nh : 0.f;
  const float tk = on ? Bk / dg : 0.f;
  double ab2[2] = {(double)tk, (double)(nh * tk)};
  cta_sumd<NM, 2>(ab2, scr);
  const float mean2 = (float)(ab2[0] / m), ny2 = (float)ab2[1];
  const float Zk = on ? (tk - mean2) - ny2 * nh : 0.f;
  double rn[2] = {(double)(Bk * Zk), (double)(Bk * Bk)};
  cta_sumd<NM, 2>(rn, scr);
  const int ld = s.ld;
  if (on) {
    kcol<float>(s.Bv, c, ld)[i] = Bk;
    kcol<float>(s.X, c, ld)[i] = 0.f;
    kcol<float>(s.R, c, ld)[i] = Bk;
    kcol<float>(s.P, c, ld)[i] = Zk;
  }
  if (threadIdx.x == 0) {
    s.rz[c] = rn[0];
    s.rhsn[c] = sqrt(rn[1]);
    s.si[SI_ACT + c] = rn[1] > 0.0 ? 1 : 0;
    s.si[SI_CITS + c] = 0;
  }
  return Bk;
}

// First-round setup of the small-face block, column c = blockIdx.x <= K of
// instance blockIdx.y, one face coordinate per thread, from G_F (gram, row
// stride NM): G nuhat, diag G, nuhat^T G nuhat and 1_F^T G 1_F, the Jacobi
// floor and lambda of k_pcg_setup
// (CTA 0 writes SD_LAM, diag G and the FP32 face data kf on F), and the start
// of column c (k_probe_fill and k_pcg_setup_cols on F; probes from the same
// counter-based generator).  Every other coordinate of these vectors is
// never read while the faces stay small.
template <int NM>
__global__ void __launch_bounds__(NM) k_face_setup(Inst base, const int* fl_base, const float* gram) {
  const int b = blockIdx.y, c = blockIdx.x;
  Inst s = inst_at(base, b);
  int* SI = s.si;
  if (SI[SI_DONE] != 0 || SI[SI_SKIPDIR] != 0 || c > SI[SI_PROBES]) return;
  const int m = SI[SI_FCNT];
  if (m > NM) return;
  __shared__ float nhs[NM];
  __shared__ double scr[NM / 32][2];
  const int k = threadIdx.x, ld = s.ld;
  const bool on = k < m;
  const int* fl = fl_base + (size_t)b * s.vs;
  const int i = on ? fl[k] : 0;
  const double nhd = on ? s.nuhat[i] : 0.0;
  const float nh = (float)nhd;
  nhs[k] = nh;
  __syncthreads();
  const float* Gm = gram + (size_t)b * NM * NM;
  // G nuhat and the sums of lambda on the right-hand side's CTA only; every
  // CTA takes the diagonal for the Jacobi floor
  float gv = 0.f, g1 = 0.f, gd = 0.f;
  if (c == 0) {  // column k of the symmetric G_F, l ascending, 32 rows of G_F staged at a time
    __shared__ float gch[32 * NM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l0 = 0; l0 < m; l0 += 32) {
      const int rows = m - l0 < 32 ? m - l0 : 32;
      for (int r = warp; r < rows; r += NM / 32)
        for (int j = lane; j < m; j += 32) cp_async4(gch + r * NM + j, Gm + (size_t)(l0 + r) * NM + j);
      cp_async_commit();
      cp_async_wait<0>();
      __syncthreads();
      if (on)
        for (int r = 0; r < rows; ++r) {
          const float gk = gch[r * NM + k];
          gv = fmaf(gk, nhs[l0 + r], gv);
          g1 += gk;
        }
      __syncthreads();
    }
  }
  if (on) gd = Gm[(size_t)k * NM + k];
  const double md = (double)SI[SI_M];
  double dd[2] = {on ? (double)gd : 0.0, on ? fabs((double)gd) : 0.0};
  cta_sumd<NM, 2>(dd, scr);
  const double floor_ = 1e-300 + 1e-12 * (dd[1] / md);
  const double dgd = on ? fmax(fabs((double)gd), floor_) : 1.0;
  if (c == 0) {
    const double T = (double)s.T, invT = s.sd[SD_INVT];
    double q4[2] = {(double)(nh * gv), (double)g1};
    cta_sumd<NM, 2>(q4, scr);
    const double psum0 = (T * q4[0]) * invT, psum1 = (T * q4[1]) * invT;  // nu^T G nu, 1_F^T G 1_F
    const double trG = dd[0] - psum1 / md - psum0;
    if (on) {
      s.diagG[i] = dgd;
      s.kf[i] = 1.f;
      s.kf[ld + i] = nh;
      s.kf[2 * (size_t)ld + i] = (float)dgd;
    }
    if (threadIdx.x == 0) s.sd[SD_LAM] = s.sd[SD_REG] * fabs(trG) / (md - 2.0);
  }
  float v = gv;
  if (c > 0 && on) {
    const unsigned long long seed =
        ((unsigned long long)(unsigned)SI[SI_SEEDHI] << 32) | (unsigned long long)(unsigned)SI[SI_SEEDLO];
    v = probe_value_f(seed, SI[SI_ITER], c - 1, i);
  }
  face_col_start<NM>(s, c, on, i, v, nh, (float)dgd, md, scr);
}

// Upper triangle of a symmetric m x m matrix in shared memory: row i from
// its diagonal at word start(i) (element (i, j), j >= i, at start(i) + j - i),
// start(0) = 0 and start(i + 1) the first word >= start(i) + m - i that is
// congruent to 2 (i + 1) mod 32.  Then, for a fixed j, threads i (= 32
// consecutive rows) reading (min(i, j), max(i, j)) hit 32 distinct banks:
// start(j) + i - j for i > j, start(i) + j - i = 2i + j (mod 32) for i <= j.
// Words used for m rows.
__host__ __device__ constexpr int face_tri_words(int m) {
  int st = 0;
  for (int i = 0; i < m; ++i) {
    const int nx = st + (m - i);
    st = nx + (((2 * (i + 1) - nx) % 32) + 32) % 32;
  }
  return st;
}
__host__ __device__ constexpr int face_tri_max_words(int nm) {
  int w = 0;
  for (int m = 1; m <= nm; ++m) w = face_tri_words(m) > w ? face_tri_words(m) : w;
  return w;
}
// Shared-memory words of k_pcg_round_small<NM>: the full matrix of any face
// of at most NM coordinates when that fits in the upper triangle's space of
// the widest block, else that space.
template <int NM>
__host__ __device__ constexpr int face_gram_words() {
  return NM * (NM + 1) <= face_tri_max_words(kMF) ? NM * (NM + 1) : face_tri_max_words(NM);
}

// A whole PCG round of column c = c0 + blockIdx.x of instance blockIdx.y on
// its face (m <= NM coordinates, one per thread), with G_F in shared memory:
// the full matrix (rows m + 1 words apart) when it fits, else the upper
// triangle in the layout above (the full matrix of a 320-coordinate face does
// not fit): the recurrence of the batched step (k_pcg_step_f) with Q = G_F p
// instead of the tensor-core products, from the state k_pcg_setup_cols (or
// k_pcg_setup2) left (X = 0, R = B, P = Z, rz, rhsn, active flag), up to the
// iteration budget; the final X, R, P and rz are written back on the face.
template <int NM>
__global__ void __launch_bounds__(NM) k_pcg_round_small(Inst base, int c0, int kmaxit, const int* fl_base,
                                                        const float* gram, int assemble) {
  const int b = blockIdx.y, c = c0 + blockIdx.x;
  Inst s = inst_at(base, b);
  int* SI = s.si;
  if (SI[SI_DONE] != 0 || SI[SI_SKIPDIR] != 0) return;
  const int m = SI[SI_FCNT];
  if (m > NM) return;
  if (SI[SI_ACT + c] == 0) {
    if (assemble) face_assemble<NM>(s, fl_base, c, 0.f);
    return;
  }
  extern __shared__ float gs[];  // upper triangle of G_F: element (i, j) at rs[i] + j (j >= i)
  __shared__ float pv[NM];
  __shared__ int rs[NM];
  __shared__ float scr[NM / 32][6];
  const int* fl = fl_base + (size_t)b * s.vs;
  const float* Gm = gram + (size_t)b * NM * NM;
  // faces whose full matrix fits (rows m + 1 words apart: distinct banks)
  // keep it; larger ones keep the upper triangle
  const bool full = m * (m + 1) <= face_gram_words<NM>();
  if (full) {
    if (threadIdx.x < m) rs[threadIdx.x] = threadIdx.x * (m + 1);
  } else if (threadIdx.x == 0) {
    int st = 0;
    for (int i = 0; i < m; ++i) {
      rs[i] = st - i;
      const int nx = st + (m - i);
      st = nx + (((2 * (i + 1) - nx) % 32) + 32) % 32;
    }
  }
  __syncthreads();
  {  // G_F into shared memory: one warp per row, every copy in flight at once
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < m; r += NM / 32)
      for (int j = (full ? 0 : r) + lane; j < m; j += 32) cp_async4(gs + rs[r] + j, Gm + (size_t)r * NM + j);
    cp_async_commit();
    cp_async_wait<0>();
  }
  const int ld = s.ld, k = threadIdx.x;
  const bool on = k < m;
  const int i = on ? fl[k] : 0;
  float* X = kcol<float>(s.X, c, ld);
  float* R = kcol<float>(s.R, c, ld);
  float* P = kcol<float>(s.P, c, ld);
  const Face<float> f0 = face_of<float>(s);
  float p = 0.f, r = 0.f, x = 0.f, nh = 0.f, dg = 1.f;
  if (on) {
    p = P[i];
    r = R[i];
    x = X[i];
    nh = f0.nh[i];
    dg = f0.dg[i];
  }
  const float mf = on ? 1.f : 0.f;
  const float fm = (float)m, lam = (float)s.sd[SD_LAM];
  const double ktol = s.sd[SD_KTOL] * s.rhsn[c];
  float rz = (float)s.rz[c];
  int its = SI[SI_CITS + c], act = 1;
  while (act) {
    pv[k] = p;
    __syncthreads();
    float q = 0.f;
    if (on) {  // q_k = sum_l G[k][l] p_l, l ascending
      const float* gr = gs + rs[k];
      if (full) {
        for (int l = 0; l < m; ++l) q = fmaf(gr[l], pv[l], q);
      } else {  // (l, k) from row l below the diagonal, (k, l) from row k
        for (int l = 0; l < k; ++l) q = fmaf(gs[rs[l] + k], pv[l], q);
        for (int l = k; l < m; ++l) q = fmaf(gr[l], pv[l], q);
      }
    }
    float a6[6] = {mf * q, nh * q, p * mf * q, p * mf, p * nh, p * p};
    cta_sum6<NM>(a6, scr);
    const float qmean = a6[0] / fm, ry = a6[1];
    const float pq = a6[2] - qmean * a6[3] - ry * a6[4] + lam * a6[5];
    if (!(pq > 0.f)) {
      act = 0;
      break;
    }
    const float al = rz / pq;
    const float qq = mf * (q - qmean) - ry * nh + lam * p;
    x += al * p;
    r -= al * qq;
    const float t = r / dg;
    float b6[6] = {r * r, mf * t, nh * t, r * mf * t, r * mf, r * nh};
    cta_sum6<NM>(b6, scr);
    its += 1;
    if (sqrt((double)b6[0]) <= ktol) {
      act = 0;
      break;
    }
    const float tmean = b6[1] / fm, tb2 = b6[2];
    const float rzn = b6[3] - tmean * b6[4] - tb2 * b6[5];
    const float beta = rzn / rz;
    p = mf * (t - tmean) - tb2 * nh + beta * p;
    rz = rzn;
    if (its >= kmaxit) {
      act = 0;
      break;
    }
    __syncthreads();  // pv is rewritten at the top of the next step
  }
  if (on) {
    X[i] = x;
    R[i] = r;
    P[i] = p;
  }
  if (threadIdx.x == 0) {
    atomicAdd(&SI[SI_KRY], its - SI[SI_CITS + c]);
    SI[SI_CITS + c] = its;
    SI[SI_ACT + c] = 0;
    s.rz[c] = (double)rz;
  }
  if (assemble) face_assemble<NM>(s, fl_base, c, x);
}

// The Hutchinson correction at = T^-1 (sum over the nchunk partials, in
// chunk order) on the face, then the second round's column ca from it: B =
// P_V at and the start of the column (k_face_hutch_finish followed by
// k_pcg_setup2, restricted to F; nchunk = 0 gives at = 0).  One CTA of NM
// threads per instance.
template <int NM>
__global__ void __launch_bounds__(NM) k_face_setup2(Inst base, const int* fl_base, const float* ap, int nchunk, int ca,
                                                    int group) {
  const int b = blockIdx.y;
  Inst s = inst_at(base, b);
  int* SI = s.si;
  if (SI[SI_DONE] != 0 || SI[SI_SKIPDIR] != 0) return;
  const int m = SI[SI_FCNT];
  if (m > NM) return;
  __shared__ double scr[NM / 32][2];
  const int k = threadIdx.x;
  const bool on = k < m;
  const int* fl = fl_base + (size_t)b * s.vs;
  const int i = on ? fl[k] : 0;
  float v = 0.f;
  if (on) {
    float a = 0.f;
    for (int c = 0; c < nchunk; ++c) a += ap[((size_t)b * nchunk + c) * NM + k];
    v = (float)(s.sd[SD_INVT] * (double)a);
  }
  const Face<float> f = face_of<float>(s);
  const float nh = on ? f.nh[i] : 0.f, dg = on ? f.dg[i] : 1.f;
  face_col_start<NM>(s, ca, on, i, v, nh, dg, (double)SI[SI_M], scr);
  if (threadIdx.x == 0) {
    SI[SI_LIVE + group] = SI[SI_ACT + ca];
    SI[SI_THIRD] += 1;
  }
}

// Partial Hutchinson corrections on the tensor cores.  CTA (x, b) covers
// rows [x kHRows, (x + 1) kHRows) of instance b in tiles of kHT = 128 rows:
// with w_2k = X_{1+k}, w_2k+1 = B_{1+k} (the PCG solutions and projected
// probes on the face, k < K <= 8), u_t = a_t W (2K values), rhat_t = K^-1
// sum_k u_t,2k u_t,2k+1, s_t = psi3(z_t) rhat_t (psi3 the third derivative of
// psi), and out[l] = sum_t s_t a_tl.  Both contractions read one staged tile
// of the face columns: coordinate l's 128 rows (AUT row upos[fl[l]],
// contiguous in t) as two 128-byte swizzled rows, one in each half tile of 64
// rows, so that the tile is
//   * MN-major for U = A_F W (M = 128 rows t, K = face coordinates l, 8-row
//     l groups 1024 bytes apart, the second half of t one half tile further):
//     D1[t][q] = sum_l a_tl W[q][l] with W split into BF16 parts (columns
//     0..15 Whi, 16..31 Wlo), and
//   * K-major for out = A_F^T s (M = 128 coordinates, K = 128 rows t):
//     D2[l][n] += sum_t a_tl S[n][t], S rows 0 and 1 the BF16 parts of s.
// FP32 accumulation in TMEM; the tile's copies are cp.async 16-byte
// transfers one tile ahead (zero-filled past the padded row end); thread 0
// issues the MMAs, threads 0..127 (one TMEM lane each) form s.  Waits are
// bounded (err |= kErrWaitTimeout on expiry).  Out: ap[(b * nchunk + x) * NM + l].
constexpr int kHT = 128;      // rows of A per tile (M of the row products, K of the back-projection)
constexpr int kHRows = 1024;  // rows of A per CTA
template <int NM>
struct HutchTc {
  static_assert(NM % 64 == 0, "face rows staged in whole 8-row atoms, weights in 64-coordinate blocks");
  static constexpr int kHalf = NM * 128;             // bytes of a half tile: 64 rows t of each of NM coordinates
  static constexpr int kStage = 2 * kHalf;           // one staged tile
  static constexpr int kWBytes = (NM / 64) * 4096;   // W: per 64 coordinates, 32 rows (Whi, Wlo) x 128 bytes
  static constexpr int kSBytes = 2 * 2048;           // S: per half tile, 16 rows x 128 bytes
  static constexpr int kMT = (NM + 127) / 128;       // M tiles of the back-projection
  static constexpr size_t kSmem = 1024 + 2 * (size_t)kStage + kWBytes + 2 * kSBytes;
  static constexpr int kMinBlocks = NM <= kMFt ? 2 : 1;
};
constexpr int kHutchChunks(long long T) { return (int)((T + kHRows - 1) / kHRows); }


// Shared-memory matrix descriptor of an MN-major tile with 128-byte swizzle:
// 64 consecutive MN elements per 128-byte row, 8 K rows per 1024-byte atom,
// K atoms 1024 bytes apart, the next 64 MN elements mn_stride bytes further.
__device__ __forceinline__ uint64_t umma_desc_sw128_mn(const void* tile, uint32_t mn_stride) {
  const uint32_t a = smem_u32(tile);
  uint64_t d = 0;
  d |= (uint64_t)((a >> 4) & 0x3FFFu);
  d |= (uint64_t)((mn_stride >> 4) & 0x3FFFu) << 16;  // leading byte offset: between 64-element MN blocks
  d |= (uint64_t)(1024 >> 4) << 32;                   // stride byte offset: between 8-row K atoms
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

template <int NM>
__global__ void __launch_bounds__(256, HutchTc<NM>::kMinBlocks)
    k_face_hutch(Inst base, int K, const int* fl_base, const __nv_bfloat16* AUT, long long ldt, const int* upos,
                 float* ap, int* err) {
  using H = HutchTc<NM>;
  const int b = blockIdx.y;
  const Inst s = inst_at(base, b);
  if (s.si[SI_DONE] != 0 || s.si[SI_SKIPDIR] != 0) return;
  const int m = s.si[SI_FCNT];
  if (m > NM || m <= 0) return;
  const long long T = s.T, t0 = (long long)blockIdx.x * kHRows;
  const long long t1 = t0 + kHRows < T ? t0 + kHRows : T;
  if (t0 >= t1) return;  // uniform over the CTA, before any barrier or TMEM use
  const int ntile = (int)((t1 - t0 + kHT - 1) / kHT);
  extern __shared__ unsigned char hsm_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(hsm_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = sm;                         // [2] staged tiles
  unsigned char* sW = sm + 2 * H::kStage;         // W (B operand of the row products)
  unsigned char* sS = sW + H::kWBytes;            // [2] S (B operand of the back-projection)
  __shared__ __align__(8) uint64_t bar[4];        // u_done, a_free[2], fin
  __shared__ uint32_t tslot;
  __shared__ int col[NM];
  __shared__ int s_abort;
  uint64_t* u_done = &bar[0];
  uint64_t* a_free = &bar[1];
  uint64_t* fin = &bar[3];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int* fl = fl_base + (size_t)b * s.vs;
  const int ld = s.ld, K2 = 2 * K, m16 = (m + 15) & ~15;
  for (int l = tid; l < NM; l += 256) col[l] = l < m ? upos[fl[l]] : 0;
  // W in BF16 parts: row q < 16 the rounding of w_q, row 16 + q that of the rest
  for (int e = tid; e < NM * 16; e += 256) {
    const int l = e >> 4, q = e & 15;
    float v = 0.f;
    if (l < m && q < K2) v = kcol<float>((q & 1) ? s.Bv : s.X, 1 + (q >> 1), ld)[fl[l]];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    unsigned char* blk = sW + (l >> 6) * 4096;
    const int jj = (l & 63) >> 3, ee = l & 7;
    *reinterpret_cast<__nv_bfloat16*>(blk + sw128_off(q, jj) + 2 * ee) = hi;
    *reinterpret_cast<__nv_bfloat16*>(blk + sw128_off(16 + q, jj) + 2 * ee) = lo;
  }
  // rows m .. m16 of both tiles enter the row products (K = m16): zero them
  // once (the copies write rows < m only); S rows 2..15 stay zero
  for (int e = tid; e < 2 * 2 * (m16 - m) * 8; e += 256) {
    const int st = e / (2 * (m16 - m) * 8), r = e - st * 2 * (m16 - m) * 8;
    const int h = r / ((m16 - m) * 8), rr = r - h * (m16 - m) * 8;
    const int l = m + (rr >> 3), jj = rr & 7;
    *reinterpret_cast<uint4*>(sA + st * H::kStage + h * H::kHalf + sw128_off(l, jj)) = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int e = tid; e < 2 * H::kSBytes / 16; e += 256) reinterpret_cast<uint4*>(sS)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) mbar_init(&bar[q], 1);
    fence_barrier_init();
    s_abort = 0;
  }
  if (warp == 0) tmem_alloc(&tslot, 128);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;  // columns 0..31 D1, 32 + 16 mt D2 of M tile mt
  const float c3 = (float)s.sd[SD_C3], c4 = (float)s.sd[SD_C4], invK = 1.f / (float)K;
  // the copies of tile i into stage i & 1: chunk c = (coordinate l, half h, 16-byte piece j)
  auto stage_tile = [&](int i) {
    unsigned char* dst = sA + (i & 1) * H::kStage;
    const long long tb = t0 + (long long)i * kHT;
    for (int c = tid; c < m * 16; c += 256) {
      const int l = c >> 4, h = (c >> 3) & 1, jj = c & 7;
      const long long t = tb + 64 * h + 8 * jj;
      const bool in = t < ldt;
      const __nv_bfloat16* src = AUT + (size_t)col[l] * ldt + (in ? t : 0);
      cp_async16(dst + h * H::kHalf + sw128_off(l, jj), src, in);
    }
    cp_async_commit();
  };
  const uint32_t id1 = idesc_bf16_f32(kTcBM, 32) | (1u << 15);  // A MN-major
  const uint32_t id2 = idesc_bf16_f32(kTcBM, 16);
  bool bad = false;
  stage_tile(0);
  // z of this thread's row of the current tile (threads < 128), loaded a tile ahead
  auto z_of = [&](int it) {
    const long long t = t0 + (long long)it * kHT + tid;
    return (tid < kHT && it < ntile && t < t1) ? (float)s.z[t] : 0.f;
  };
  float zc = z_of(0);
  int i = 0;
  for (; i < ntile; ++i) {
    const int st = i & 1;
    const float zn = z_of(i + 1);
    if (i >= 1 && !mbar_wait_bounded(&a_free[st ^ 1], (uint32_t)(((i - 1) >> 1) & 1))) bad = true;
    if (i + 1 < ntile) stage_tile(i + 1);
    else cp_async_commit();  // an empty group keeps the count
    cp_async_wait<1>();      // the copies of tile i are done
    fence_proxy_async_smem();
    if (bad) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    unsigned char* pa = sA + st * H::kStage;
    if (tid == 0) {
      tc_fence_after();
      for (int kk = 0; kk < m16 / 16; ++kk) {
        const uint64_t da = umma_desc_sw128_mn(pa + kk * 2048, (uint32_t)H::kHalf);
        const uint64_t dw = umma_desc_sw128(sW + (kk >> 2) * 4096 + (kk & 3) * 32);
        umma_bf16(tmem, da, dw, id1, kk > 0 ? 1u : 0u);
      }
      umma_commit(u_done);
    }
    unsigned char* ps = sS + st * H::kSBytes;
    if (warp < 4) {
      if (!mbar_wait_bounded(u_done, (uint32_t)(i & 1))) bad = true;
      tc_fence_after();
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
      float rh = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) rh = fmaf(v[2 * k] + v[16 + 2 * k], v[2 * k + 1] + v[17 + 2 * k], rh);
      const long long t = t0 + (long long)i * kHT + tid;
      float sv = 0.f;
      if (t < t1) sv = (-6.f * c3 + 24.f * c4 * zc) * (rh * invK);
      const __nv_bfloat16 hi = __float2bfloat16_rn(sv);
      const __nv_bfloat16 lo = __float2bfloat16_rn(sv - __bfloat162float(hi));
      const int h = tid >> 6, jj = (tid & 63) >> 3, ee = tid & 7;
      *reinterpret_cast<__nv_bfloat16*>(ps + h * 2048 + sw128_off(0, jj) + 2 * ee) = hi;
      *reinterpret_cast<__nv_bfloat16*>(ps + h * 2048 + sw128_off(1, jj) + 2 * ee) = lo;
      fence_proxy_async_smem();
      tc_fence_before();
    }
    if (bad) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int mt = 0; mt < H::kMT; ++mt) {
        const int r0 = mt * 128 < NM - 128 ? mt * 128 : NM - 128;  // the last M tile ends at row NM
        if (mt * 128 >= m) break;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int h = kk >> 2;
          const uint64_t da = umma_desc_sw128(pa + h * H::kHalf + (r0 >> 3) * 1024 + (kk & 3) * 32);
          const uint64_t ds = umma_desc_sw128(ps + h * 2048 + (kk & 3) * 32);
          umma_bf16(tmem + 32u + 16u * mt, da, ds, id2, (i > 0 || kk > 0) ? 1u : 0u);
        }
      }
      umma_commit(&a_free[st]);
    }
    zc = zn;
  }
  cp_async_wait<0>();
  if (tid == 0) umma_commit(fin);  // arrives once every MMA issued above has completed
  const bool ok = mbar_wait_bounded(fin, 0);
  if (!ok && tid == 0) atomicOr(err, kErrWaitTimeout);
  if (s_abort && tid == 0) atomicOr(err, kErrWaitTimeout);
  tc_fence_after();
  if (ok && !s_abort && warp < 4) {
#pragma unroll
    for (int mt = 0; mt < H::kMT; ++mt) {
      const int r0 = mt * 128 < NM - 128 ? mt * 128 : NM - 128;
      if (mt * 128 >= m) break;
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 32u + 16u * mt, v);
      const int l = r0 + tid;
      if (l >= mt * 128 && l < m) ap[((size_t)b * gridDim.x + blockIdx.x) * NM + l] = v[0] + v[1];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// at_b = T^-1 sum over the chunks (fixed order) on the face, zero elsewhere.
template <int NM>
__global__ void k_face_hutch_finish(Inst base, const int* fl_base, const float* ap, int nchunk) {
  const int b = blockIdx.x;
  Inst s = inst_at(base, b);
  if (s.si[SI_DONE] != 0 || s.si[SI_SKIPDIR] != 0) return;
  const int m = s.si[SI_FCNT];
  if (m > NM) return;
  const int* fl = fl_base + (size_t)b * s.vs;
  for (int i = threadIdx.x; i < s.ld; i += blockDim.x) s.at[i] = 0.0;
  __syncthreads();
  const double invT = s.sd[SD_INVT];
  for (int l = threadIdx.x; l < m; l += blockDim.x) {
    float v = 0.f;
    for (int c = 0; c < nchunk; ++c) v += ap[((size_t)b * nchunk + c) * NM + l];
    s.at[fl[l]] = invT * (double)v;
  }
}
