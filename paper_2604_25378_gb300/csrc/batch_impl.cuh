// Lockstep batched PCG YAND-MVSK solve (included into mvsk_api.cu).
//
// B independent instances (lambda_b, target_b) on the same A advance together:
// every iteration is one captured graph in which
//   * the FP64 value/gradient and line-search passes run per instance,
//   * the affine-normal blocks of all instances share the tensor-core
//     products (all instances' PCG columns side by side in one N dimension),
//   * the O(n) kernels run one CTA per instance (grid.y = instance).
// Each instance carries a host state machine for the stall-recovery phases
// and the return-target calibration (the same sequence of solves, c1 values
// and warm starts as mvsk_solve).  Instances that are done skip every kernel.
#pragma once

// ---------------------------------------------------------------- kernels
// Batches keep their Krylov vectors in FP32 (see the PCG kernels), so these
// kernels use no FP64 arithmetic per element.
// dst[(b*nc + j)*ld + i] = bf16(col_j of instance b): PCG column c0 + j, or the
// interleaved (X_{1+k}, B_{1+k}) pairs when interleave != 0.  Grid
// (ld/1024, B*nc): four coordinates per thread (ld is a multiple of 64, so the
// 16-byte loads and 8-byte stores are aligned).
__global__ void k_cols_bf16_b(Inst base, int nc, int c0, int interleave, __nv_bfloat16* dst) {
  const int ld = base.ld;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i >= ld) return;
  const int q = blockIdx.y, b = q / nc, j = q % nc;
  const Inst s = inst_at(base, b);
  const float* col = interleave ? ((j & 1) ? kcol<float>(s.Bv, 1 + (j >> 1), ld) : kcol<float>(s.X, 1 + (j >> 1), ld))
                                : kcol<float>(s.P, c0 + j, ld);
  const float4 v = *reinterpret_cast<const float4*>(col + i);
  __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
  uint2 pk;
  pk.x = *reinterpret_cast<uint32_t*>(&lo);
  pk.y = *reinterpret_cast<uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(dst + (size_t)q * ld + i) = pk;
}

// S^T[q][t] = bf16(h_b[t] * sum_z part[z][q][t]), b = q / nc, with
// h_b = psi''_b(z_b) in FP32 (k_hd_reduce1).  Grid (ceil(T / 1024), N): four
// consecutive rows per thread, with 16-byte loads and one 8-byte store when
// T is a multiple of 4 (rows then start 16-byte aligned; Tp is a multiple of 8).
__global__ void k_reduce_hvp1_b(const float* part, int splits, int N, int nc, long long T, long long ldp,
                                const float* Hf, __nv_bfloat16* S, long long Tp, const int* rts = nullptr) {
  const long long t0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (t0 >= T) return;
  if (rts != nullptr) splits = rts[2];
  const int q = blockIdx.y;
  const float* h = Hf + (size_t)(q / nc) * T;
  __nv_bfloat16* out = S + (size_t)q * Tp;
  if ((T & 3) == 0 && (ldp & 3) == 0) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int z = 0; z < splits; ++z) {
      const float4 v = *reinterpret_cast<const float4*>(part + ((size_t)z * N + q) * ldp + t0);
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    const float4 hv = *reinterpret_cast<const float4*>(h + t0);
    __nv_bfloat162 lo = __floats2bfloat162_rn(hv.x * acc.x, hv.y * acc.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn(hv.z * acc.z, hv.w * acc.w);
    uint2 pk;
    pk.x = *reinterpret_cast<uint32_t*>(&lo);
    pk.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(out + t0) = pk;
    return;
  }
  for (long long t = t0; t < t0 + 4 && t < T; ++t) {
    float acc = 0.f;
#pragma unroll 4
    for (int z = 0; z < splits; ++z) acc += part[((size_t)z * N + q) * ldp + t];
    out[t] = __float2bfloat16(h[t] * acc);
  }
}

// at_b = T^-1 sum_z part[z][b][i] (FP64 output: the back-projected correction).
// With upos (face-restricted products) the partial row of coordinate i is
// upos[i] (< 0: outside the union of the faces, value 0) and the split count
// rts[2] is the runtime one.
__global__ void k_reduce_at_b(const float* part, int splits, int B, int n, int ld, long long ldp, double scale,
                              Inst base, const int* rts = nullptr, const int* upos = nullptr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ld) return;
  const int b = blockIdx.y;
  const Inst s = inst_at(base, b);
  if (rts != nullptr) splits = rts[2];
  const int row = i < n ? (upos != nullptr ? upos[i] : i) : -1;
  float acc = 0.f;
  if (row >= 0)
#pragma unroll 4
    for (int z = 0; z < splits; ++z) acc += part[((size_t)z * B + b) * ldp + row];
  s.at[i] = scale * (double)acc;
}

// rhat_b[t] = K^-1 sum_k (A X_k)_t (A p_k)_t; S^T[b][t] = bf16(psi3_b(z_b[t]) rhat_b[t]).
// Grid (T/256, B).  The pair products come from BF16 operands, so FP32 sums of
// K of them lose nothing; only the BF16 weights are kept (the lockstep path has
// no other reader of rhat).
__global__ void k_reduce_rhat_b(const float* part, int splits, int N, int K, long long T, long long ldp, Inst base,
                                __nv_bfloat16* S, long long Tp, const int* rts = nullptr) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (t >= T) return;
  if (rts != nullptr) splits = rts[2];
  const Inst s = inst_at(base, b);
  float r = 0.f;
  for (int k = 0; k < K; ++k) {
    float u = 0.f, v = 0.f;
    const int q = b * 2 * K + 2 * k;
    for (int z = 0; z < splits; ++z) {
      u += part[((size_t)z * N + q) * ldp + t];
      v += part[((size_t)z * N + q + 1) * ldp + t];
    }
    r = fmaf(u, v, r);
  }
  const Psi psi{0.0, s.sd[SD_C3], s.sd[SD_C4]};
  const float w = (float)psi.d3(s.z[t]);
  S[(size_t)b * Tp + t] = __float2bfloat16(w * (r / (float)K));
}

// ------------------------------------------- split tensor-core FP64 products
// Finishing kernels of the split products of ozaki.cuh for instances
// b0 .. b0 + gridDim.y - 1 (local index = blockIdx.y = column of the product).
// Row kernels stride over t with gridDim.x CTAs; CTA g writes its scalar
// partials to spart_b[g * ns + q], the layout the single-CTA kernels reduce.

// z_b = A x_b (Prop. 1, z_t = a_t^T w); W_b = psi'_b(z_b); spart_b[g] = sum psi_b(z_t).
// Runs only when *needz != 0: otherwise z_b is the cache that k_z_step keeps.
__global__ void __launch_bounds__(256) k_oz_fin_z(const long long* part, int splits, int Bp, long long ldp,
                                                  const int* em, const int* fb, Inst base, int b0, double* W,
                                                  long long ldw, const int* needz) {
  __shared__ double scr[64];
  if (*needz == 0) return;
  const int bl = blockIdx.y;
  Inst s = inst_at(base, b0 + bl);
  if (s.si[SI_DONE] != 0) return;
  const Psi psi{s.sd[SD_C2], s.sd[SD_C3], s.sd[SD_C4]};
  double acc = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < s.T; t += (long long)gridDim.x * blockDim.x) {
    const double z = oz_value(part, splits, Bp, ldp, t, bl, em[t], fb[bl]);
    s.z[t] = z;
    W[(size_t)(b0 + bl) * ldw + t] = psi.d1(z);
    acc += psi.f(z);
  }
  acc = block_sum(acc, scr);
  if (threadIdx.x == 0) s.spart[blockIdx.x] = acc;
}

// The value terms from the cached z_b (when *needz == 0): W_b = psi'_b(z_b) and
// spart_b[g] = sum psi_b(z_t) over the rows of CTA g, the layout of k_oz_fin_z.
// The cache follows every step: A(x + alpha d) = z + alpha A d (proof of
// Prop. 3), with A d the line-search product of the step (k_z_step); inner
// solves start from the cached A 1/n or the cached z of their warm start.
__global__ void __launch_bounds__(256) k_z_fin(Inst base, int b0, double* W, long long ldw, const int* needz) {
  __shared__ double scr[64];
  if (*needz != 0) return;
  const int bl = blockIdx.y;
  Inst s = inst_at(base, b0 + bl);
  if (s.si[SI_DONE] != 0) return;
  const Psi psi{s.sd[SD_C2], s.sd[SD_C3], s.sd[SD_C4]};
  double acc = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < s.T; t += (long long)gridDim.x * blockDim.x) {
    const double z = s.z[t];
    W[(size_t)(b0 + bl) * ldw + t] = psi.d1(z);
    acc += psi.f(z);
  }
  acc = block_sum(acc, scr);
  if (threadIdx.x == 0) s.spart[blockIdx.x] = acc;
}

// z_b += alpha_b w_b, w_b = A d_b stored by the line-search finish, for the
// instances whose step took that direction: phase 1 after k_decide1 (raw or
// capped step along d), phase 2 after k_decide2 (the segment or face hand-off,
// SKIPLS == 0).  Coordinates moved onto tau by the step's clamp (within
// eps_act = 1e-15) are not followed.  Grid (Gz, B).
__global__ void __launch_bounds__(256) k_z_step(Inst base, const double* wls, int phase) {
  const int b = blockIdx.y;
  Inst s = inst_at(base, b);
  if (s.si[SI_DONE] != 0) return;
  if (phase == 1) {
    const int br = s.si[SI_BRANCH];
    if (br != BR_RAW && br != BR_CAPPED) return;
  } else if (s.si[SI_SKIPLS] != 0) {
    return;
  }
  const double al = s.sd[SD_ALPHA];
  if (al == 0.0) return;
  const double* w = wls + (size_t)b * s.T;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < s.T; t += (long long)gridDim.x * blockDim.x)
    s.z[t] += al * w[t];
}

// g_b = -c1_b mu + T^-1 A^T psi'_b(z_b) (Eq. operator-grad), zero padding to ld.
__global__ void k_oz_fin_g(const long long* part, int splits, int Bp, long long ldp, const int* em, const int* fb,
                           Inst base, int b0) {
  const int bl = blockIdx.y;
  Inst s = inst_at(base, b0 + bl);
  if (s.si[SI_DONE] != 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.ld) return;
  s.g[i] = i < s.n ? -s.sd[SD_C1] * s.mu[i] + s.sd[SD_INVT] * oz_value(part, splits, Bp, ldp, i, bl, em[i], fb[bl])
                   : 0.0;
}

// The twelve power sums s_rs of (z_t, w_t = a_t^T d) (Prop. quartic line search).
// w_b[t] (the projected direction) is also stored in wout[(b0 + b) * T + t]
// for the cache update of z (k_z_step).
// kinfo (nullable): the product ran on a coordinate list of padded length
// kinfo[1]; its slot count is then oz_slots(kinfo[1] / 64).
__global__ void __launch_bounds__(256) k_oz_fin_ls(const long long* part, int splits, int Bp, long long ldp,
                                                   const int* em, const int* fb, Inst base, int b0, int skip_slot,
                                                   double* wout, const int* kinfo = nullptr,
                                                   const int* need = nullptr) {
  __shared__ double red[9][256];
  if (need != nullptr && *need == 0) return;  // the product did not run
  const int bl = blockIdx.y;
  if (kinfo != nullptr) splits = oz_slots(kinfo[1] / kTcBK);
  Inst s = inst_at(base, b0 + bl);
  if (s.si[SI_DONE] != 0 || s.si[skip_slot] != 0) return;
  // the nine sums with w: the z-only sums s20, s30, s40 enter no quartic
  // coefficient (Prop. quartic line search) and are written as zero
  double a[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) a[q] = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < s.T; t += (long long)gridDim.x * blockDim.x) {
    const double zt = s.z[t], w = oz_value(part, splits, Bp, ldp, t, bl, em[t], fb[bl]);
    wout[(size_t)(b0 + bl) * s.T + t] = w;
    const double z2 = zt * zt, w2 = w * w;
    a[0] += zt * w;        // s11
    a[1] += z2 * w;        // s21
    a[2] += z2 * zt * w;   // s31
    a[3] += w2;            // s02
    a[4] += zt * w2;       // s12
    a[5] += z2 * w2;       // s22
    a[6] += w2 * w;        // s03
    a[7] += zt * w2 * w;   // s13
    a[8] += w2 * w2;       // s04
  }
  // Staged reduction of the nine sums: 16 threads per sum add 16 values
  // each, then a 16-lane shuffle tree (two barriers instead of one tree and
  // two barriers per sum).
#pragma unroll
  for (int q = 0; q < 9; ++q) red[q][threadIdx.x] = a[q];
  __syncthreads();
  if (threadIdx.x < 160) {  // whole warps in the shuffles; lanes of q = 9 add zeros
    const int q = threadIdx.x >> 4, j = threadIdx.x & 15;
    double v = 0.0;
    if (q < 9)
#pragma unroll
      for (int k = 0; k < 16; ++k) v += red[q][j + 16 * k];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (j == 0 && q < 9) s.spart[(size_t)blockIdx.x * 12 + 3 + q] = v;
  } else if (threadIdx.x < 163) {
    s.spart[(size_t)blockIdx.x * 12 + (threadIdx.x - 160)] = 0.0;
  }
}

// g = -c1 mu + G0 (the gradient at 1/n from its c1-free part), zero padding.
__global__ void k_grad_from_g0(double* g, const double* G0, const double* mu, double c1, int n, int ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ld) g[i] = i < n ? -c1 * mu[i] + G0[i] : 0.0;
}

// KKT residual at the 1/n start of the inner solves of instances idx[j]
// (grid.y = j), the kkt_rel normaliser: g(1/n) = -c1_j mu + G0_b.  Scratch:
// instance columns 18 (g) and 19 (x = 1/n) of tmp.
__global__ void __launch_bounds__(kVT) k_kkt0_batch(Inst base, const int* idx, const double* c1, const double* G0) {
  __shared__ double scr[80];
  const int b = idx[blockIdx.y];
  Inst s = inst_at(base, b);
  const int n = s.n, ld = s.ld;
  double* g = s.tmp + (size_t)18 * ld;
  double* x = s.tmp + (size_t)19 * ld;
  const double cj = c1[blockIdx.y];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    g[i] = -cj * s.mu[i] + G0[(size_t)b * ld + i];
    x[i] = 1.0 / n;
  }
  __syncthreads();
  const double k0 = kkt_residual(x, g, n, s.sd[SD_TAU], scr, s.tmp);
  if (threadIdx.x == 0) s.sd[SD_KKT0] = k0;
}

// w[t] = psi'(z[t]) with coefficients (c2, c3, c4), t < T.
__global__ void k_dpsi_into(const double* z, long long T, double c2, double c3, double c4, double* w) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < T) w[t] = Psi{c2, c3, c4}.d1(z[t]);
}

// Second line-search product, over the running instances that take the
// projected segment (SKIPLS == 0): need[0] = 1 when it runs on all columns of
// A, need[1] = 1 when it runs on the union of the working faces (umode, and
// every such segment vanishes off the union: SI_LS2OUT == 0).
__global__ void k_need_ls2(Inst base, int B, int* need, int umode) {
  int any = 0, out = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int* si = base.si + (size_t)b * kSI;
    const int take = si[SI_DONE] == 0 && si[SI_SKIPLS] == 0;
    any |= take;
    out |= take && (umode == 0 || si[SI_LS2OUT] != 0);
  }
  any = __syncthreads_or(any);
  out = __syncthreads_or(out);
  if (threadIdx.x == 0) {
    need[0] = out;
    need[1] = any && !out;
  }
}

// ------------------------------------- diagonal and nu-products (tensor cores)
// The per-iteration inputs of the PCG block (Sec. 3.2): G nu and diag(G) of
// the weighted Gram G = T^-1 A^T Diag(psi''(z)) A, plus psi''-weighted squares
// of A nu and A 1_F (traces of the face-projected Hessian), for all instances.

// dst[(2b + j)*ld + i] = bf16(nuhat_b[i]) (j = 0) or bf16(maskF_b[i]) (j = 1).
__global__ void k_hd_cols(Inst base, int B, __nv_bfloat16* dst) {
  const int ld = base.ld;
  const long long tot = (long long)B * 2 * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % ld);
    const long long q = e / ld;
    const Inst s = inst_at(base, (int)(q >> 1));
    dst[e] = __float2bfloat16((float)((q & 1) ? s.maskF[i] : s.nuhat[i]));
  }
}

// From the split partials of A [nu_b, 1_F,b]: h = psi''_b(z_t), S^T[b][t] =
// bf16(h (A nu)_t), H[b][t] = bf16(h), Hf[b][t] = h in FP32 (reused by the
// PCG products of the iteration); spart_b[g*2 + {0,1}] = sum h (A nu)_t^2,
// sum h (A 1_F)_t^2 over the rows t of CTA g.
__global__ void __launch_bounds__(256) k_hd_reduce1(const float* part, int splits, int N, long long T, long long ldp,
                                                    Inst base, __nv_bfloat16* S, __nv_bfloat16* H, long long Tp,
                                                    float* Hf, const int* rts = nullptr) {
  __shared__ double scr[64];
  const int b = blockIdx.y;
  Inst s = inst_at(base, b);
  if (s.si[SI_SKIPDIR] != 0) return;
  if (rts != nullptr) splits = rts[2];
  // psi'' in FP32 (its consumers are FP32 and BF16); FP64 only for the sums
  const float c2 = (float)s.sd[SD_C2], c3 = (float)s.sd[SD_C3], c4 = (float)s.sd[SD_C4];
  double a0 = 0.0, a1 = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (long long)gridDim.x * blockDim.x) {
    float u = 0.f, v = 0.f;
#pragma unroll 4
    for (int z = 0; z < splits; ++z) {
      u += part[((size_t)z * N + 2 * b) * ldp + t];
      v += part[((size_t)z * N + 2 * b + 1) * ldp + t];
    }
    const float zt = (float)s.z[t];
    const float h = 2.f * c2 - zt * (6.f * c3 - 12.f * c4 * zt);
    S[(size_t)b * Tp + t] = __float2bfloat16(h * u);
    H[(size_t)b * Tp + t] = __float2bfloat16(h);
    Hf[(size_t)b * T + t] = h;
    a0 += (double)(h * u * u);
    a1 += (double)(h * v * v);
  }
  a0 = block_sum(a0, scr);
  a1 = block_sum(a1, scr);
  if (threadIdx.x == 0) {
    s.spart[(size_t)blockIdx.x * 2] = a0;
    s.spart[(size_t)blockIdx.x * 2 + 1] = a1;
  }
}

// out_b[i] = T^-1 sum_z part[z][b][i] into Gnu_b (which = 0) or diagG_b (which = 1).
// upos / rts: as in k_reduce_at_b.
__global__ void k_hd_reduce2(const float* part, int splits, int B, int n, int ld, long long ldp, double scale,
                             Inst base, int which, const int* rts = nullptr, const int* upos = nullptr) {
  const long long tot = (long long)B * ld;
  if (rts != nullptr) splits = rts[2];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / ld), i = (int)(e % ld);
    const Inst s = inst_at(base, b);
    if (s.si[SI_SKIPDIR] != 0) continue;
    const int row = i < n ? (upos != nullptr ? upos[i] : i) : -1;
    double acc = 0.0;
    if (row >= 0)
      for (int z = 0; z < splits; ++z) acc += (double)part[((size_t)z * B + b) * ldp + row];
    (which ? s.diagG : s.Gnu)[i] = scale * acc;
  }
}

// out[j*ldo + t] = bf16(A[t*lda + j]^2) for j < n, t < T; zero for T <= t < Tp.
__global__ void k_square_t_bf16(const double* A, int lda, long long T, int n, __nv_bfloat16* out, long long ldo,
                                long long Tp) {
  __shared__ float tile[32][33];
  const long long t0 = (long long)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const long long t = t0 + threadIdx.y + 8 * k;
    const int j = j0 + threadIdx.x;
    double v = 0.0;
    if (t < T && j < n) v = A[(size_t)t * lda + j];
    tile[threadIdx.y + 8 * k][threadIdx.x] = (float)(v * v);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = j0 + threadIdx.y + 8 * k;
    const long long t = t0 + threadIdx.x;
    if (j < n && t < Tp) out[(size_t)j * ldo + t] = __float2bfloat16(tile[threadIdx.x][threadIdx.y + 8 * k]);
  }
}

// Split-K count for `tiles` output tiles of nk k-blocks on `slots` resident
// CTAs.  Tensor-bound tiles: the count minimising waves * (k-blocks per split)
// + 6 per split (prologue, epilogue and partial traffic in k-block units).
// Bandwidth-bound tiles: one wave of resident CTAs, so every SM streams A at
// once.  At least 4 k-blocks per split, at most smax splits.
__host__ __device__ inline int pick_splits(int tiles, int nk, int slots, bool tensor_bound, int smax) {
  if (!tensor_bound) {
    int sp = slots / tiles;
    if (sp > smax) sp = smax;
    if (sp > nk / 4) sp = nk / 4;
    return sp < 1 ? 1 : sp;
  }
  int best = 1;
  long long best_cost = -1;
  for (int sp = 1; sp <= smax; ++sp) {
    if (sp > 1 && nk < 4 * sp) break;
    const long long waves = ((long long)tiles * sp + slots - 1) / slots;
    const long long cost = waves * ((nk + sp - 1) / sp) + 6LL * sp;
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = sp;
    }
  }
  return best;
}


// --------------------------------------------- face-restricted products (U)
// After the face step every PCG vector of instance b lives on its working
// face F_b (zero elsewhere), so A v reads only the columns of A in F_b and
// the back-projection A^T s is needed only on F_b.  Per iteration the union U
// of the running instances' faces (|U| is a few hundred once the faces have
// collapsed, against n = 5440) is listed, the columns of A in U are gathered
// in both orientations, and the direction products run with K = |U| (A P) or
// |U| output rows (A^T S): the same sums over fewer zero terms.
//
// Runtime extents of the products: one spec per product launch (filled at
// graph capture), completed per iteration by k_union_scan.
constexpr int kUMaxProds = 16;
constexpr int kUMaxSplits = 16;

// flag[i] = 1 when coordinate i is on the working face of a running
// instance (k_face wrote maskF this iteration); the direction d of every
// running instance, trivial faces included, is zero off its face.
__global__ void k_union_flags(Inst base, int B, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= base.ld) return;
  int f = 0;
  if (i < base.n) {
    // independent loads (no early exit), so that they are all in flight at once
#pragma unroll 8
    for (int b = 0; b < B; ++b) {
      // mask != 0 tested on the bits (integer pipe): nonzero apart from the sign
      const long long mb = __double_as_longlong(base.maskF[(size_t)b * base.vs + i]);
      f |= (int)(base.si[(size_t)b * kSI + SI_DONE] == 0) & (int)((mb << 1) != 0);
    }
  }
  flag[i] = f;
}

// One CTA of 1024 threads: U in increasing order (idx[j], j < |U|), the
// position of each coordinate in it (pos[i], -1 outside), info[0] = |U|,
// info[1] = |U| rounded up to 64 (at least 64), and the runtime extents
// rt[4 p .. 4 p + 3] = {rows, K, splits, k-tiles per split} of product spec p
// (every split non-empty, as the consumers sum that many partials).
__global__ void __launch_bounds__(1024) k_union_scan(const int* flag, int ld, int* idx, int* pos, int* info,
                                                     const UProd* specs, int nspec, int* rt) {
  __shared__ int wsum[32];
  const int per = (ld + 1023) / 1024, i0 = threadIdx.x * per;
  int cnt = 0;
  for (int i = i0; i < i0 + per && i < ld; ++i) cnt += flag[i];
  // exclusive scan of cnt over the block
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
  for (int i = i0; i < i0 + per && i < ld; ++i) {
    if (flag[i]) {
      idx[p] = i;
      pos[i] = p++;
    } else {
      pos[i] = -1;
    }
  }
  if (threadIdx.x == 1023) {
    const int ku = p, kup = ku < 1 ? kTcBK : (ku + kTcBK - 1) / kTcBK * kTcBK;
    info[0] = ku;
    info[1] = kup;
    for (int q = 0; q < nspec; ++q) {
      const UProd& sp = specs[q];
      if (sp.mrows <= 0 || sp.nt <= 0) continue;  // unused slot
      const int rows = sp.rows_dyn ? kup : sp.M, K = sp.rows_dyn ? sp.K : kup;
      const int mt = (rows + sp.mrows - 1) / sp.mrows, nk = (K + kTcBK - 1) / kTcBK;
      const int want = pick_splits(mt * sp.nt, nk, sp.slots, sp.tensor != 0, sp.smax);
      const int ktps = (nk + want - 1) / want;
      rt[4 * q] = rows;
      rt[4 * q + 1] = K;
      rt[4 * q + 2] = (nk + ktps - 1) / ktps;
      rt[4 * q + 3] = ktps;
    }
  }
}

// dst row j = src row idx[j] for j < |U|, zero for |U| <= j < info[1]
// (rows of cols BF16 values, cols a multiple of 8).  Grid (x, rows of dst).
__global__ void k_gather_rows_bf16(const __nv_bfloat16* __restrict__ src, long long lds, const int* idx,
                                   const int* info, __nv_bfloat16* __restrict__ dst, long long ldd, long long cols) {
  const int j = blockIdx.y;
  if (j >= info[1]) return;
  const bool live = j < info[0];
  const uint4* s4 = reinterpret_cast<const uint4*>(src + (size_t)(live ? idx[j] : 0) * lds);
  uint4* d4 = reinterpret_cast<uint4*>(dst + (size_t)j * ldd);
  const long long n8 = cols / 8;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n8; e += (long long)gridDim.x * blockDim.x)
    d4[e] = live ? s4[e] : make_uint4(0u, 0u, 0u, 0u);
}

// dst[t][j] = srcT[j][t] for j < info[1], t < T (64 x 64 tiles through
// shared memory; dst is T x ldd, srcT is rows x lds).  Grid (ceil(T/64),
// ceil(rows/64)), block (64, 8).
__global__ void k_transpose_u_bf16(const __nv_bfloat16* __restrict__ srcT, long long lds, const int* info,
                                   long long T, __nv_bfloat16* __restrict__ dst, long long ldd) {
  __shared__ __nv_bfloat16 tile[64][66];
  const int j0 = blockIdx.y * 64;
  if (j0 >= info[1]) return;
  const long long t0 = (long long)blockIdx.x * 64;
  for (int r = threadIdx.y; r < 64; r += 8) {
    const long long t = t0 + threadIdx.x;
    tile[r][threadIdx.x] = t < T ? srcT[(size_t)(j0 + r) * lds + t] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 64; r += 8) {
    const long long t = t0 + r;
    if (t < T) dst[(size_t)t * ldd + j0 + threadIdx.x] = tile[threadIdx.x][r];
  }
}

// BF16 columns in U coordinates: dst[q*ld + j] = bf16(col_q[idx[j]]) for
// j < |U|, zero for |U| <= j < info[1]; col_q as in k_cols_bf16_b.
__global__ void k_cols_bf16_u(Inst base, int nc, int c0, int interleave, const int* idx, const int* info,
                              __nv_bfloat16* dst) {
  const int ld = base.ld;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= info[1]) return;
  const int q = blockIdx.y, b = q / nc, jj = q % nc;
  const Inst s = inst_at(base, b);
  const float* col = interleave ? ((jj & 1) ? kcol<float>(s.Bv, 1 + (jj >> 1), ld) : kcol<float>(s.X, 1 + (jj >> 1), ld))
                                : kcol<float>(s.P, c0 + jj, ld);
  dst[(size_t)q * ld + j] = __float2bfloat16(j < info[0] ? col[idx[j]] : 0.f);
}

// The nuhat / maskF columns of the Gram-diagonal block in U coordinates.
__global__ void k_hd_cols_u(Inst base, const int* idx, const int* info, __nv_bfloat16* dst) {
  const int ld = base.ld;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= info[1]) return;
  const int q = blockIdx.y;
  const Inst s = inst_at(base, q >> 1);
  float v = 0.f;
  if (j < info[0]) v = (float)((q & 1) ? s.maskF[idx[j]] : s.nuhat[idx[j]]);
  dst[(size_t)q * ld + j] = __float2bfloat16(v);
}

#include "face_small.cuh"

// ---------------------------------------------------------------- host side

mvsk_status batch_alloc(mvsk_ctx* c, BatchBuf& bb, int B) {
  if (bb.cap >= B) return MVSK_OK;
  for (void* q : bb.mem) cudaFree(q);
  bb.mem.clear();
  bb.cap = 0;
  const size_t ld = (size_t)c->ld, T = (size_t)c->T, nc = (size_t)c->ncolmax;
  auto get = [&](size_t bytes, void** p) -> mvsk_status {
    cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(MVSK_ENOMEM, "batch allocation of %zu bytes failed", bytes);
    }
    bb.mem.push_back(*p);
    CU(cudaMemsetAsync(*p, 0, bytes < 16 ? 16 : bytes, c->stream));
    return MVSK_OK;
  };
  Inst s{};
  void* p;
  const size_t Bs = (size_t)B;
#define GETD(field, count)                        \
  TRY(get(sizeof(double) * (count), &p));         \
  s.field = (double*)p
  TRY(get(sizeof(double) * kSD * Bs, &p));
  s.sd = (double*)p;
  TRY(get(sizeof(int) * kSI * Bs, &p));
  s.si = (int*)p;
  s.mu = c->mu;
  GETD(x, ld * Bs);
  GETD(g, ld * Bs);
  GETD(nuhat, ld * Bs);
  GETD(maskF, ld * Bs);
  GETD(d, ld * Bs);
  GETD(dstep, ld * Bs);
  GETD(xbar, ld * Bs);
  GETD(at, ld * Bs);
  GETD(bestx, ld * Bs);
  TRY(get(sizeof(double) * 2 * ld * Bs, &p));
  s.Gnu = (double*)p;
  s.diagG = s.Gnu + ld;
  GETD(tmp, ld * (nc + 4) * Bs);
  GETD(z, T * Bs);
  GETD(rhat, T * Bs);
  GETD(X, ld * nc * Bs);
  GETD(R, ld * nc * Bs);
  GETD(Zc, ld * nc * Bs);
  GETD(P, ld * nc * Bs);
  GETD(Q, ld * nc * Bs);
  GETD(Bv, ld * nc * Bs);
  GETD(rz, nc * Bs);
  GETD(rhsn, nc * Bs);
  GETD(spart, (size_t)16 * c->grid * Bs);
#undef GETD
  s.n = c->n;
  s.ld = c->ld;
  s.T = c->T;
  s.vs = c->ld;
  s.ts = c->T;
  s.cs = (long long)c->ld * c->ncolmax;
  s.ps = (long long)c->ld * (c->ncolmax + 4);
  s.ncs = c->ncolmax;
  s.ss = 16LL * c->grid;
  bb.base = s;
  TRY(ensure_tc_operands(c));
  TRY(get(sizeof(__nv_bfloat16) * kTcCols * ld * Bs, &p));
  bb.P16 = (__nv_bfloat16*)p;
  TRY(get(sizeof(__nv_bfloat16) * kTcCols * (size_t)c->Tp * Bs, &p));
  bb.S16T = (__nv_bfloat16*)p;
  bb.part_floats = (size_t)4 * kTcCols * Bs * (T > ld ? T : ld);
  TRY(get(sizeof(float) * bb.part_floats, &p));
  bb.part = (float*)p;
  TRY(get(sizeof(double) * T * Bs, &p));
  bb.Wt = (double*)p;
  TRY(get(sizeof(int) * 4, &p));
  bb.need = (int*)p;
  TRY(get(sizeof(double) * ld * Bs, &p));
  bb.G0 = (double*)p;
  TRY(get(sizeof(double) * T * Bs, &p));
  bb.wls = (double*)p;
  TRY(get(sizeof(double) * 2 * T * Bs, &p));
  bb.zsave = (double*)p;
  TRY(get(sizeof(double) * T, &p));
  bb.z0 = (double*)p;
  TRY(get(sizeof(int), &p));
  bb.needz = (int*)p;
  TRY(get(sizeof(__nv_bfloat16) * (size_t)c->Tp * Bs, &p));
  bb.H16 = (__nv_bfloat16*)p;
  TRY(get(sizeof(float) * T * Bs, &p));
  bb.Hf = (float*)p;
  TRY(get(sizeof(float) * 3 * ld * Bs, &p));
  bb.base.kf = (float*)p;
  bb.base.kfs = 3LL * c->ld;
  TRY(get(sizeof(double) * 2 * Bs, &p));
  bb.kq_dev = p;
  {  // small-face direction block
    const size_t nch = (size_t)kHutchChunks(c->T);
    TRY(get(sizeof(int) * ld * Bs, &p));
    bb.f_list = (int*)p;
    TRY(get(sizeof(float) * kGramSplit * kMF * kMF * Bs, &p));  // partial Grams, one slab per share of T
    bb.f_gp = (float*)p;
    TRY(get(sizeof(float) * kMF * kMF * Bs, &p));
    bb.f_gram = (float*)p;
    TRY(get(sizeof(float) * nch * kMF * Bs, &p));
    bb.f_ap = (float*)p;
  }
  if (c->A2_16T == nullptr) {
    TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * (size_t)c->n * c->Tp));
    c->A2_16T = (__nv_bfloat16*)p;
    dim3 g((unsigned)((c->Tp + 31) / 32), (unsigned)((c->n + 31) / 32));
    k_square_t_bf16<<<g, dim3(32, 8), 0, c->stream>>>(c->A64, c->ld, c->T, c->n, c->A2_16T, c->Tp, c->Tp);
    c->launches += 1;
    CU(cudaGetLastError());
  }
  bb.cap = B;
  return MVSK_OK;
}

// N tile and resident CTAs per SM of the batched products.  Wide products
// take the tile among 128, 192 and 256 that pads N least (ties: the wider),
// since padded columns still cost full MMA work.
inline int tc_bn(int N) {
  if (N <= 16) return 16;
  if (N <= 64) return 64;
  int best = 256, waste = 1 << 30;
  for (int bn : {256, 192, 128}) {
    const int w = (N + bn - 1) / bn * bn - N;
    if (w < waste) {
      waste = w;
      best = bn;
    }
  }
  return best;
}
inline int tc_ctas_per_sm(int bn) { return bn == 64 ? 2 : 1; }
inline bool tc_wide(int bn) { return bn >= 128; }

// Launch of the two-subtile (256-row) product with N tile bn and epilogue epi.
template <class Epi>
void launch_tc2(int bn, dim3 grid, cudaStream_t st, const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K,
                int ktps, const Epi& epi, int* err, const int* rt = nullptr) {
  if (bn == 128)
    k_gemm_tc<128, 4, Epi, 2><<<grid, 128, tc_smem_bytes<128, 4, 2>(), st>>>(ta, tb, M, N, K, ktps, epi, err,
                                                                            nullptr, nullptr, rt);
  else if (bn == 192)
    k_gemm_tc<192, 4, Epi, 2><<<grid, 128, tc_smem_bytes<192, 4, 2>(), st>>>(ta, tb, M, N, K, ktps, epi, err,
                                                                            nullptr, nullptr, rt);
  else
    k_gemm_tc<256, 3, Epi, 2><<<grid, 128, tc_smem_bytes<256, 3, 2>(), st>>>(ta, tb, M, N, K, ktps, epi, err,
                                                                            nullptr, nullptr, rt);
}

// Split-K tensor-core product with FP32 partials for N columns (N tile 16, 64 or 256).
template <class Epi>
void launch_partials(int bn, dim3 grid, cudaStream_t st, const CUtensorMap& ta, const CUtensorMap& tb, int M, int N,
                     int K, int ktps, const Epi& epi, int* err, const int* rt = nullptr) {
  if (bn == 16)
    k_gemm_tc<16, 8, Epi><<<grid, 128, tc_smem_bytes<16, 8>(), st>>>(ta, tb, M, N, K, ktps, epi, err, nullptr,
                                                                     nullptr, rt);
  else if (bn == 64)
    k_gemm_tc<64, 4, Epi><<<grid, 128, tc_smem_bytes<64, 4>(), st>>>(ta, tb, M, N, K, ktps, epi, err, nullptr,
                                                                     nullptr, rt);
  else
    launch_tc2(bn, grid, st, ta, tb, M, N, K, ktps, epi, err, rt);
}

mvsk_status tc_partials_n(mvsk_ctx* c, const void* Aop, int M, const void* Bop, int N, long long K, long long ldk,
                          float* part, size_t part_floats, long long ldp, int* splits_out) {
  CUtensorMap ta, tb;
  const int bn = tc_bn(N);
  TRY(make_tmap_bf16(&ta, Aop, (unsigned long long)ldk, (unsigned long long)M, (unsigned long long)ldk * 2, kTcBK,
                     kTcBM));
  TRY(make_tmap_bf16(&tb, Bop, (unsigned long long)ldk, (unsigned long long)N, (unsigned long long)ldk * 2, kTcBK,
                     (unsigned)bn));
  const int mrows = tc_wide(bn) ? 2 * kTcBM : kTcBM;  // wide N tiles: two 128-row subtiles per CTA
  const int mt = (M + mrows - 1) / mrows, nt = (N + bn - 1) / bn;
  const int nk = (int)((K + kTcBK - 1) / kTcBK);
  int smax = (int)(part_floats / ((size_t)N * ldp));
  if (smax > 8) smax = 8;
  if (smax < 1) smax = 1;
  const int want = pick_splits(mt * nt, nk, c->nsm * tc_ctas_per_sm(bn), tc_wide(bn), smax);
  const int ktps = (nk + want - 1) / want;
  const int splits = (nk + ktps - 1) / ktps;
  dim3 grid((unsigned)nt, (unsigned)mt, (unsigned)splits);
  TRY(prof_begin(c, 400 + bn, 2.0 * (double)M * (double)N * (double)K));
  if ((ldp * 4) % 16 == 0) {  // partials through bulk tensor stores (box of 32 rows x CW columns)
    const cuuint64_t dims[3] = {(cuuint64_t)M, (cuuint64_t)N, (cuuint64_t)splits};
    const cuuint64_t strides[2] = {(cuuint64_t)ldp * 4, (cuuint64_t)N * (cuuint64_t)ldp * 4};
    const cuuint32_t box[3] = {32, (cuuint32_t)(bn < 32 ? bn : 32), 1};
    EpiPartTma epi;
    TRY(make_tmap_store(&epi.tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, part, dims, strides, box));
    launch_partials(bn, grid, c->stream, ta, tb, M, N, (int)K, ktps, epi, c->err);
  } else {
    const EpiPartT epi{part, ldp, M, N};
    launch_partials(bn, grid, c->stream, ta, tb, M, N, (int)K, ktps, epi, c->err);
  }
  c->launches += 1;
  CU(cudaGetLastError());
  TRY(prof_end(c));
  *splits_out = splits;
  return MVSK_OK;
}

// Hessian-vector products of PCG columns c0..c0+nc of every instance, up to
// the split partials of A^T S (the PCG step sums them):
// S^T = bf16(psi''(z) o A P16) from the first product, fused into its
// epilogue when it needs no split-K.  P16 holds the BF16 columns already.
// *fused (nullable) tells which form the first product took: 1 the fused
// weighting epilogue, 0 split-K partials and k_reduce_hvp1_b.
mvsk_status hvp_tc_batch(mvsk_ctx* c, BatchBuf& bb, int B, int nc, int* s2, int* fused = nullptr) {
  const int N = B * nc;
  const unsigned gt4 = (unsigned)((c->T + 1023) / 1024);
  const int bn = tc_bn(N), mt = (int)((c->T + 2 * kTcBM - 1) / (2 * kTcBM)), nt = (N + bn - 1) / bn;
  const int nk = (int)((c->ld + kTcBK - 1) / kTcBK);
  const bool fuse = tc_wide(bn) && 2 * mt * nt >= c->nsm;
  if (fused != nullptr) *fused = fuse ? 1 : 0;
  if (fuse) {  // enough work without split-K: fuse the weighting
    CUtensorMap ta, tb;
    TRY(make_tmap_bf16(&ta, c->Alo, (unsigned long long)c->ld, (unsigned long long)c->T,
                       (unsigned long long)c->ld * 2, kTcBK, kTcBM));
    TRY(make_tmap_bf16(&tb, bb.P16, (unsigned long long)c->ld, (unsigned long long)N, (unsigned long long)c->ld * 2,
                       kTcBK, (unsigned)bn));
    // S^T through bulk tensor stores: map {T, N} (rows T <= t < Tp stay zero), box {32, 32}
    EpiHvp1Tma epi;
    epi.Hf = bb.Hf;
    epi.T = (int)c->T;
    epi.N = N;
    epi.nc = nc;
    const cuuint64_t dims[2] = {(cuuint64_t)c->T, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)c->Tp * 2};
    const cuuint32_t box[2] = {32, 32};
    TRY(make_tmap_store(&epi.tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, bb.S16T, dims, strides, box));
    TRY(prof_begin(c, 400 + bn, 2.0 * (double)c->T * (double)N * (double)c->ld));
    launch_tc2(bn, dim3((unsigned)nt, (unsigned)mt, 1), c->stream, ta, tb, (int)c->T, N, c->ld, nk, epi, c->err);
    c->launches += 1;
    CU(cudaGetLastError());
    TRY(prof_end(c));
  } else {
    int s1 = 0;
    TRY(tc_partials_n(c, c->Alo, (int)c->T, bb.P16, N, c->ld, c->ld, bb.part, bb.part_floats, c->T, &s1));
    PROF_LAUNCH(NK_HVP1, (k_reduce_hvp1_b<<<dim3(gt4, N), 256, 0, c->stream>>>(bb.part, s1, N, nc, c->T, c->T, bb.Hf,
                                                                               bb.S16T, c->Tp)));
  }
  return tc_partials_n(c, c->A16T, c->n, bb.S16T, N, c->Tp, c->Tp, bb.part, bb.part_floats, c->ld, s2);
}

// rhat_b and at_b = T^-1 A^T (psi3_b(z_b) o rhat_b) for every instance.
mvsk_status third_tc_batch(mvsk_ctx* c, BatchBuf& bb, int B, int K) {
  const int N = B * 2 * K;
  const unsigned gl = (unsigned)((c->ld + 255) / 256), gl4 = (unsigned)((c->ld + 1023) / 1024);
  PROF_LAUNCH(NK_COLS, (k_cols_bf16_b<<<dim3(gl4, N), 256, 0, c->stream>>>(bb.base, 2 * K, 0, 1, bb.P16)));
  int s1 = 0, s2 = 0;
  TRY(tc_partials_n(c, c->Alo, (int)c->T, bb.P16, N, c->ld, c->ld, bb.part, bb.part_floats, c->T, &s1));
  PROF_LAUNCH(NK_RHAT, (k_reduce_rhat_b<<<dim3((unsigned)((c->T + 255) / 256), B), 256, 0, c->stream>>>(bb.part, s1, N, K, c->T, c->T, bb.base, bb.S16T,
                                                                   c->Tp)));
  TRY(tc_partials_n(c, c->A16T, c->n, bb.S16T, B, c->Tp, c->Tp, bb.part, bb.part_floats, c->ld, &s2));
  PROF_LAUNCH(NK_HVP2, (k_reduce_at_b<<<dim3(gl, B), 256, 0, c->stream>>>(bb.part, s2, B, c->n, c->ld, c->ld,
                                                                         1.0 / (double)c->T, bb.base)));
  return MVSK_OK;
}

// Gnu, diagG and the two psi''-weighted squares of every instance (skips
// instances with SI_SKIPDIR); scalar partials with gz CTAs over t.
mvsk_status hvpdiag_tc_batch(mvsk_ctx* c, BatchBuf& bb, int B, int gz) {
  const int N = 2 * B, gb = 4 * c->nsm;
  PROF_LAUNCH(NK_HD_COLS, (k_hd_cols<<<gb, 256, 0, c->stream>>>(bb.base, B, bb.P16)));
  int s1 = 0, s2 = 0, s3 = 0;
  TRY(tc_partials_n(c, c->Alo, (int)c->T, bb.P16, N, c->ld, c->ld, bb.part, bb.part_floats, c->T, &s1));
  PROF_LAUNCH(NK_HD_RED1, (k_hd_reduce1<<<dim3(gz, B), 256, 0, c->stream>>>(bb.part, s1, N, c->T, c->T, bb.base,
                                                                            bb.S16T, bb.H16, c->Tp, bb.Hf)));
  TRY(tc_partials_n(c, c->A16T, c->n, bb.S16T, B, c->Tp, c->Tp, bb.part, bb.part_floats, c->ld, &s2));
  PROF_LAUNCH(NK_HD_RED2, (k_hd_reduce2<<<gb, 256, 0, c->stream>>>(bb.part, s2, B, c->n, c->ld, c->ld,
                                                                   1.0 / (double)c->T, bb.base, 0)));
  TRY(tc_partials_n(c, c->A2_16T, c->n, bb.H16, B, c->Tp, c->Tp, bb.part, bb.part_floats, c->ld, &s3));
  PROF_LAUNCH(NK_HD_DIAG, (k_hd_reduce2<<<gb, 256, 0, c->stream>>>(bb.part, s3, B, c->n, c->ld, c->ld,
                                                                   1.0 / (double)c->T, bb.base, 1)));
  return MVSK_OK;
}

// ------------------------------------------ face-restricted products (host)
// Spec slot of a product shape (find or add); the specs are uploaded before the
// first replay of the graph and k_union_scan fills their runtime extents.
int u_spec(BatchBuf& bb, const UProd& p) {
  for (size_t q = 0; q < bb.u_hspec.size(); ++q) {
    const UProd& o = bb.u_hspec[q];
    if (o.rows_dyn == p.rows_dyn && o.M == p.M && o.K == p.K && o.mrows == p.mrows && o.nt == p.nt &&
        o.slots == p.slots && o.tensor == p.tensor && o.smax == p.smax)
      return (int)q;
  }
  bb.u_hspec.push_back(p);
  return (int)bb.u_hspec.size() - 1;
}

// Spec of a product restricted to U (see UProd); fused: the psi''-weighted
// A P without split-K.
UProd u_shape(const mvsk_ctx* c, int rows_dyn, int Mmax, int N, long long K, size_t part_floats, long long ldp,
              bool fused) {
  const int bn = tc_bn(N);
  const int mrows = tc_wide(bn) ? 2 * kTcBM : kTcBM;
  const int nt = (N + bn - 1) / bn;
  int smax = fused ? 1 : (int)(part_floats / ((size_t)N * ldp));
  if (smax > kUMaxSplits) smax = kUMaxSplits;
  if (smax < 1) smax = 1;
  return UProd{rows_dyn, rows_dyn ? 0 : Mmax, rows_dyn ? (int)K : 0, mrows, nt,
               c->nsm * (fused ? 1 : tc_ctas_per_sm(bn)), tc_wide(bn) ? 1 : 0, smax};
}

bool u_fused(const mvsk_ctx* c, int N) {
  const int bn = tc_bn(N), mt = (int)((c->T + 2 * kTcBM - 1) / (2 * kTcBM)), nt = (N + bn - 1) / bn;
  return tc_wide(bn) && 2 * mt * nt >= c->nsm;
}

// Every product shape a lockstep iteration (or a parity export) launches on U,
// registered and uploaded before any of them runs: the Gram-diagonal block,
// the Hessian-vector blocks of widths nc[0..nw), the Hutchinson block of K
// probe pairs (K = 0: none).
mvsk_status u_prepare(mvsk_ctx* c, BatchBuf& bb, int B, const int* nc, int nw, int K) {
  bb.u_hspec.clear();
  const size_t pf = bb.part_floats;
  u_spec(bb, u_shape(c, 0, (int)c->T, 2 * B, c->ld, pf, c->T, false));
  u_spec(bb, u_shape(c, 1, c->ld, B, c->Tp, pf, c->ld, false));
  for (int w = 0; w < nw; ++w) {
    const int N = B * nc[w];
    const bool f = u_fused(c, N);
    u_spec(bb, u_shape(c, 0, (int)c->T, N, c->ld, pf, c->T, f));
    u_spec(bb, u_shape(c, 1, c->ld, N, c->Tp, pf, c->ld, false));
  }
  if (K > 0) u_spec(bb, u_shape(c, 0, (int)c->T, 2 * K * B, c->ld, pf, c->T, false));
  if (bb.u_hspec.size() > (size_t)kUMaxProds) return fail(MVSK_ECUDA, "too many face-restricted product shapes");
  std::vector<UProd> all((size_t)kUMaxProds, UProd{0, 0, 0, 0, 0, 0, 0, 0});
  for (size_t q = 0; q < bb.u_hspec.size(); ++q) all[q] = bb.u_hspec[q];
  CU(cudaMemcpyAsync(bb.u_specs, all.data(), sizeof(UProd) * kUMaxProds, cudaMemcpyHostToDevice, c->stream));
  return sync(c);
}

// Slot of a registered shape (u_prepare), -1 if it was not registered.
int u_find(const BatchBuf& bb, const UProd& p) {
  for (size_t q = 0; q < bb.u_hspec.size(); ++q) {
    const UProd& o = bb.u_hspec[q];
    if (o.rows_dyn == p.rows_dyn && o.M == p.M && o.K == p.K && o.mrows == p.mrows && o.nt == p.nt &&
        o.slots == p.slots && o.tensor == p.tensor && o.smax == p.smax)
      return (int)q;
  }
  return -1;
}

// Split-K product restricted to the union U.  rows_dyn = 0: A P with A the
// gathered T x |U| columns (K = |U|, output rows fixed); rows_dyn = 1: A^T S
// with the gathered |U| rows (output rows |U|, K fixed).  Partials as in
// tc_partials_n, with the runtime split count at (*rts_out)[2] (device).
mvsk_status tc_partials_u(mvsk_ctx* c, BatchBuf& bb, int rows_dyn, const void* Aop, int Mmax, const void* Bop, int N,
                          long long K, long long ldk, float* part, size_t part_floats, long long ldp,
                          const int** rts_out) {
  CUtensorMap ta, tb;
  const int bn = tc_bn(N);
  TRY(make_tmap_bf16(&ta, Aop, (unsigned long long)ldk, (unsigned long long)Mmax, (unsigned long long)ldk * 2, kTcBK,
                     kTcBM));
  TRY(make_tmap_bf16(&tb, Bop, (unsigned long long)ldk, (unsigned long long)N, (unsigned long long)ldk * 2, kTcBK,
                     (unsigned)bn));
  const UProd sp = u_shape(c, rows_dyn, Mmax, N, K, part_floats, ldp, false);
  const int q = u_find(bb, sp);
  if (q < 0) return fail(MVSK_ECUDA, "face-restricted product shape not registered");
  const int* rt = bb.u_rt + 4 * q;
  const int mt = (Mmax + sp.mrows - 1) / sp.mrows;
  dim3 grid((unsigned)sp.nt, (unsigned)mt, (unsigned)sp.smax);
  // profiler work: FLOPs per unit of |U| (scaled by the runtime |U| when read)
  TRY(prof_begin_u(c, 400 + bn, 2.0 * (double)N * (double)(rows_dyn ? K : Mmax)));
  if ((ldp * 4) % 16 == 0) {  // partials through bulk tensor stores
    const cuuint64_t dims[3] = {(cuuint64_t)Mmax, (cuuint64_t)N, (cuuint64_t)sp.smax};
    const cuuint64_t strides[2] = {(cuuint64_t)ldp * 4, (cuuint64_t)N * (cuuint64_t)ldp * 4};
    const cuuint32_t box[3] = {32, (cuuint32_t)(bn < 32 ? bn : 32), 1};
    EpiPartTma epi;
    TRY(make_tmap_store(&epi.tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, part, dims, strides, box));
    launch_partials(bn, grid, c->stream, ta, tb, Mmax, N, (int)K, 1, epi, c->err, rt);
  } else {  // rows of partials not 16-byte aligned (T not a multiple of 4): plain stores
    const EpiPartT epi{part, ldp, Mmax, N};
    launch_partials(bn, grid, c->stream, ta, tb, Mmax, N, (int)K, 1, epi, c->err, rt);
  }
  c->launches += 1;
  CU(cudaGetLastError());
  TRY(prof_end(c));
  *rts_out = rt;
  return MVSK_OK;
}

// Union of the faces and the gathered operands of this iteration.
mvsk_status union_gather(mvsk_ctx* c, BatchBuf& bb, int B) {
  const unsigned gl = (unsigned)((c->ld + 255) / 256);
  PROF_LAUNCH(NK_UNION, (k_union_flags<<<gl, 256, 0, c->stream>>>(bb.base, B, bb.u_flag)));
  PROF_LAUNCH(NK_UNION, (k_union_scan<<<1, 1024, 0, c->stream>>>(bb.u_flag, c->ld, bb.u_idx, bb.u_pos, bb.u_info,
                                                                  bb.u_specs, kUMaxProds, bb.u_rt)));
  const unsigned gx = (unsigned)((c->Tp / 8 + 255) / 256);
  PROF_LAUNCH(NK_GATHER, (k_gather_rows_bf16<<<dim3(gx, (unsigned)c->ld), 256, 0, c->stream>>>(
                             c->A16T, c->Tp, bb.u_idx, bb.u_info, bb.u_AUT, c->Tp, c->Tp)));
  PROF_LAUNCH(NK_GATHER, (k_transpose_u_bf16<<<dim3((unsigned)((c->T + 63) / 64), (unsigned)(c->ld / 64)), dim3(64, 8),
                                               0, c->stream>>>(bb.u_AUT, c->Tp, bb.u_info, c->T, bb.u_AU, c->ld)));
  return MVSK_OK;
}

// hvpdiag_tc_batch on the union: Gnu, diagG and the two weighted squares.
mvsk_status hvpdiag_tc_batch_u(mvsk_ctx* c, BatchBuf& bb, int B, int gz) {
  const int N = 2 * B, gb = 4 * c->nsm;
  const unsigned gl = (unsigned)((c->ld + 255) / 256);
  const unsigned gx = (unsigned)((c->Tp / 8 + 255) / 256);
  PROF_LAUNCH(NK_GATHER, (k_gather_rows_bf16<<<dim3(gx, (unsigned)c->ld), 256, 0, c->stream>>>(
                             c->A2_16T, c->Tp, bb.u_idx, bb.u_info, bb.u_A2UT, c->Tp, c->Tp)));
  PROF_LAUNCH(NK_HD_COLS, (k_hd_cols_u<<<dim3(gl, (unsigned)N), 256, 0, c->stream>>>(bb.base, bb.u_idx, bb.u_info,
                                                                                      bb.P16)));
  const int *r1 = nullptr, *r2 = nullptr, *r3 = nullptr;
  TRY(tc_partials_u(c, bb, 0, bb.u_AU, (int)c->T, bb.P16, N, c->ld, c->ld, bb.part, bb.part_floats, c->T, &r1));
  PROF_LAUNCH(NK_HD_RED1, (k_hd_reduce1<<<dim3(gz, B), 256, 0, c->stream>>>(bb.part, 1, N, c->T, c->T, bb.base,
                                                                            bb.S16T, bb.H16, c->Tp, bb.Hf, r1)));
  TRY(tc_partials_u(c, bb, 1, bb.u_AUT, c->ld, bb.S16T, B, c->Tp, c->Tp, bb.part, bb.part_floats, c->ld, &r2));
  PROF_LAUNCH(NK_HD_RED2, (k_hd_reduce2<<<gb, 256, 0, c->stream>>>(bb.part, 1, B, c->n, c->ld, c->ld,
                                                                   1.0 / (double)c->T, bb.base, 0, r2, bb.u_pos)));
  TRY(tc_partials_u(c, bb, 1, bb.u_A2UT, c->ld, bb.H16, B, c->Tp, c->Tp, bb.part, bb.part_floats, c->ld, &r3));
  PROF_LAUNCH(NK_HD_DIAG, (k_hd_reduce2<<<gb, 256, 0, c->stream>>>(bb.part, 1, B, c->n, c->ld, c->ld,
                                                                   1.0 / (double)c->T, bb.base, 1, r3, bb.u_pos)));
  return MVSK_OK;
}

// hvp_tc_batch on the union: P16 holds the columns in U coordinates; the
// partials of A^T S come out in U coordinates (*rts: their split count).
mvsk_status hvp_tc_batch_u(mvsk_ctx* c, BatchBuf& bb, int B, int nc, const int** rts) {
  const int N = B * nc;
  const unsigned gt4 = (unsigned)((c->T + 1023) / 1024);
  const int bn = tc_bn(N), mt = (int)((c->T + 2 * kTcBM - 1) / (2 * kTcBM)), nt = (N + bn - 1) / bn;
  if (u_fused(c, N)) {  // fused weighting, K = |U| at run time
    CUtensorMap ta, tb;
    TRY(make_tmap_bf16(&ta, bb.u_AU, (unsigned long long)c->ld, (unsigned long long)c->T,
                       (unsigned long long)c->ld * 2, kTcBK, kTcBM));
    TRY(make_tmap_bf16(&tb, bb.P16, (unsigned long long)c->ld, (unsigned long long)N, (unsigned long long)c->ld * 2,
                       kTcBK, (unsigned)bn));
    EpiHvp1Tma epi;
    epi.Hf = bb.Hf;
    epi.T = (int)c->T;
    epi.N = N;
    epi.nc = nc;
    const cuuint64_t dims[2] = {(cuuint64_t)c->T, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)c->Tp * 2};
    const cuuint32_t box[2] = {32, 32};
    TRY(make_tmap_store(&epi.tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, bb.S16T, dims, strides, box));
    const int q = u_find(bb, u_shape(c, 0, (int)c->T, N, c->ld, bb.part_floats, c->T, true));
    if (q < 0) return fail(MVSK_ECUDA, "face-restricted product shape not registered");
    TRY(prof_begin_u(c, 400 + bn, 2.0 * (double)c->T * (double)N));
    launch_tc2(bn, dim3((unsigned)nt, (unsigned)mt, 1), c->stream, ta, tb, (int)c->T, N, c->ld, 1, epi, c->err,
               bb.u_rt + 4 * q);
    c->launches += 1;
    CU(cudaGetLastError());
    TRY(prof_end(c));
  } else {
    const int* r1 = nullptr;
    TRY(tc_partials_u(c, bb, 0, bb.u_AU, (int)c->T, bb.P16, N, c->ld, c->ld, bb.part, bb.part_floats, c->T, &r1));
    PROF_LAUNCH(NK_HVP1, (k_reduce_hvp1_b<<<dim3(gt4, N), 256, 0, c->stream>>>(bb.part, 1, N, nc, c->T, c->T, bb.Hf,
                                                                               bb.S16T, c->Tp, r1)));
  }
  return tc_partials_u(c, bb, 1, bb.u_AUT, c->ld, bb.S16T, N, c->Tp, c->Tp, bb.part, bb.part_floats, c->ld, rts);
}

// third_tc_batch on the union.
mvsk_status third_tc_batch_u(mvsk_ctx* c, BatchBuf& bb, int B, int K) {
  const int N = B * 2 * K;
  const unsigned gl = (unsigned)((c->ld + 255) / 256);
  PROF_LAUNCH(NK_COLS, (k_cols_bf16_u<<<dim3(gl, (unsigned)N), 256, 0, c->stream>>>(bb.base, 2 * K, 0, 1, bb.u_idx,
                                                                                     bb.u_info, bb.P16)));
  const int *r1 = nullptr, *r2 = nullptr;
  TRY(tc_partials_u(c, bb, 0, bb.u_AU, (int)c->T, bb.P16, N, c->ld, c->ld, bb.part, bb.part_floats, c->T, &r1));
  PROF_LAUNCH(NK_RHAT, (k_reduce_rhat_b<<<dim3((unsigned)((c->T + 255) / 256), B), 256, 0, c->stream>>>(
                           bb.part, 1, N, K, c->T, c->T, bb.base, bb.S16T, c->Tp, r1)));
  TRY(tc_partials_u(c, bb, 1, bb.u_AUT, c->ld, bb.S16T, B, c->Tp, c->Tp, bb.part, bb.part_floats, c->ld, &r2));
  PROF_LAUNCH(NK_HVP2, (k_reduce_at_b<<<dim3(gl, B), 256, 0, c->stream>>>(bb.part, 1, B, c->n, c->ld, c->ld,
                                                                         1.0 / (double)c->T, bb.base, r2, bb.u_pos)));
  return MVSK_OK;
}

PassArgs pass_args_inst(const double cc[4]) {
  PassArgs a;
  memset(&a, 0, sizeof(a));
  a.c2 = cc[1];
  a.c3 = cc[2];
  a.c4 = cc[3];
  a.rscale = 1.0;
  return a;
}

// One lockstep iteration of every instance (captured once per batch solve).
mvsk_status batch_iteration_tail(mvsk_ctx* c, BatchBuf& bb, int B, const std::vector<std::array<double, 4>>& cc);

// Direction block of an iteration whose working faces all have at most NM
// coordinates (face_small.cuh): face Grams on the tensor cores, both PCG
// rounds in shared memory, the Hutchinson correction between them.
template <int NM>
mvsk_status small_face_direction(mvsk_ctx* c, BatchBuf& bb, int B) {
  const Inst& base = bb.base;
  const int K = c->opt.probes, ncol1 = K + 1, ca = K + 1, kmax = c->opt.krylov_maxit;
  const unsigned nch = (unsigned)kHutchChunks(c->T);
  using GT = GramTc<NM>;
  // face Grams on the tensor cores, rows of A in GT::kSplit shares per instance
  PROF_LAUNCH(NK_GRAM, (k_face_gram_tc<NM><<<dim3(GT::kSplit, B, (NM + 127) / 128), 256, GT::kSmem, c->stream>>>(
                           base, bb.f_list, bb.u_AUT, c->Tp, bb.u_pos, bb.f_gp, c->err)));
  PROF_LAUNCH(NK_GRAM_FIN, (k_face_gram_sum<NM><<<dim3(16, B), 256, 0, c->stream>>>(base, bb.f_gp, GT::kSplit,
                                                                                      bb.f_gram)));
  // every Krylov vector of both rounds lives on the face: setups on F only
  PROF_LAUNCH(NK_PCG_SETUP, (k_face_setup<NM><<<dim3(ncol1, B), NM, 0, c->stream>>>(base, bb.f_list, bb.f_gram)));
  const size_t gsm = sizeof(float) * face_gram_words<NM>();
  PROF_LAUNCH(NK_PCG_ROUND, (k_pcg_round_small<NM><<<dim3(ncol1, B), NM, gsm, c->stream>>>(base, 0, kmax, bb.f_list,
                                                                                          bb.f_gram, 0)));
  if (K > 0)
    PROF_LAUNCH(NK_HUTCH, (k_face_hutch<NM><<<dim3(nch, B), 256, HutchTc<NM>::kSmem, c->stream>>>(
                              base, K, bb.f_list, bb.u_AUT, c->Tp, bb.u_pos, bb.f_ap, c->err)));
  PROF_LAUNCH(NK_PCG_SETUP2, (k_face_setup2<NM><<<dim3(1, B), NM, 0, c->stream>>>(base, bb.f_list, bb.f_ap,
                                                                                  K > 0 ? (int)nch : 0, ca, ca / 2)));
  // the second round's CTA also assembles d on the face
  PROF_LAUNCH(NK_PCG_ROUND, (k_pcg_round_small<NM><<<dim3(1, B), NM, gsm, c->stream>>>(base, ca, kmax, bb.f_list,
                                                                                      bb.f_gram, 1)));
  return MVSK_OK;
}

// The Hutchinson correction of the small-face block alone (NM-coordinate
// launch shape), from the face lists and union gather already in place.
template <int NM>
mvsk_status small_face_third(mvsk_ctx* c, BatchBuf& bb, int B, int K) {
  const unsigned nch = (unsigned)kHutchChunks(c->T);
  PROF_LAUNCH(NK_HUTCH, (k_face_hutch<NM><<<dim3(nch, B), 256, HutchTc<NM>::kSmem, c->stream>>>(
                            bb.base, K, bb.f_list, bb.u_AUT, c->Tp, bb.u_pos, bb.f_ap, c->err)));
  PROF_LAUNCH(NK_HUTCH, (k_face_hutch_finish<NM><<<B, 256, 0, c->stream>>>(bb.base, bb.f_list, bb.f_ap, (int)nch)));
  return MVSK_OK;
}


// part -1: the whole iteration; with face-restricted products (bb.umode) it
// is captured as three graphs: part 0 the oracle block (value, gradient,
// face, face lists, union of the faces and its gathered columns), then part 2
// the small-face direction block (face_small.cuh) when every face has at most
// kMF coordinates, else part 1 (tensor-core products on the union); both end
// with the quartic step and the boundary block.
mvsk_status batch_iteration(mvsk_ctx* c, BatchBuf& bb, int B, const std::vector<std::array<double, 4>>& cc,
                            int part = -1) {
  const Inst& base = bb.base;
  const int K = c->opt.probes, ncol1 = K + 1, ca = K + 1, kmax = c->opt.krylov_maxit;
  const int P = c->dir_prec;
  const bool split = c->opt.split_products != 0;
  const OzBuf& oz = c->oz;
  const int Gz = oz_row_ctas(c);
  const int Gs = split ? Gz : c->grid;  // scalar partials per instance of the value product
  const int Gl = split ? oz_ls_ctas(c) : c->grid;  // ... and of the line-search products
  // split products of one of the directions d (d_b = base + b*vs) for groups of <= 64 instances
  auto ls_split = [&](double* dvec, int skip_slot, const int* need) -> mvsk_status {
    for (int b0 = 0; b0 < B; b0 += kOzMaxB) {
      const int nb = B - b0 < kOzMaxB ? B - b0 : kOzMaxB;
      int sp = 0;
      TRY(oz_product(c, 0, dvec + (size_t)b0 * base.vs, base.vs, nb, oz_bp(nb), need, &sp));
      PROF_LAUNCH(NK_OZ_LS, (k_oz_fin_ls<<<dim3(Gl, nb), 256, 0, c->stream>>>(oz.part, sp, oz_bp(nb), oz.MpF, oz.eF,
                                                                             oz.fF, base, b0, skip_slot, bb.wls)));
    }
    return MVSK_OK;
  };
  const bool head = part <= 0, dir = part != 0;
  if (head && split) {
    for (int b0 = 0; b0 < B; b0 += kOzMaxB) {
      const int nb = B - b0 < kOzMaxB ? B - b0 : kOzMaxB, Bp = oz_bp(nb);
      int sp = 0;
      TRY(oz_product(c, 0, base.x + (size_t)b0 * base.vs, base.vs, nb, Bp, bb.needz, &sp));
      PROF_LAUNCH(NK_OZ_Z, (k_oz_fin_z<<<dim3(Gz, nb), 256, 0, c->stream>>>(oz.part, sp, Bp, oz.MpF, oz.eF, oz.fF,
                                                                           base, b0, bb.Wt, c->T, bb.needz)));
      PROF_LAUNCH(NK_OZ_Z, (k_z_fin<<<dim3(Gz, nb), 256, 0, c->stream>>>(base, b0, bb.Wt, c->T, bb.needz)));
      TRY(oz_product(c, 1, bb.Wt + (size_t)b0 * c->T, c->T, nb, Bp, nullptr, &sp));
      PROF_LAUNCH(NK_OZ_G, (k_oz_fin_g<<<dim3((c->ld + 255) / 256, nb), 256, 0, c->stream>>>(
                                oz.part, sp, Bp, oz.MpB, oz.eB, oz.fB, base, b0)));
    }
  } else if (head) {
    for (int b = 0; b < B; ++b) {
      const Inst s = inst_at(base, b);
      PassArgs a = pass_args_inst(cc[b].data());
      a.in[0] = s.x;
      a.rowout = s.z;
      a.skip = s.si + SI_DONE;
      TRY(run_pass(c, P64, M_VALGRAD, 1, a, nullptr, s.spart));
      TRY(reduce_cols(c, P64, 1, s.g, c->ld, c->mu, 0.0, s.si + SI_DONE, nullptr, s.sd + SD_C1));
    }
  }
  const bool U = bb.umode;  // direction products restricted to the union of the faces
  if (head) {
    PROF_LAUNCH(NK_FACE, (k_face<<<dim3(1, B), kVT, 0, c->stream>>>(base, nullptr, Gs)));
    if (U) {
      PROF_LAUNCH(NK_FACE_LIST, (k_face_list<<<dim3(1, B), 1024, 0, c->stream>>>(base, bb.f_list)));
      PROF_LAUNCH(NK_FACE_LIST, (k_small_mode<<<1, 256, 0, c->stream>>>(base, B, c->opt.face_small != 0,
                                                                         c->opt.face_small == 2, bb.u_info, bb.cond,
                                                                         bb.has_cond)));
      TRY(union_gather(c, bb, B));
      if (split && bb.u_AFU != nullptr)  // digit planes of A's columns in U (the line search along d)
        PROF_LAUNCH(NK_OZ_SPLIT_U, (k_oz_split_rows_u<<<4 * c->nsm, 256, 0, c->stream>>>(
                                     c->A64, c->ld, c->T, bb.u_idx, bb.u_info, oz.eF, bb.u_AFU, oz.MpF)));
    }
  }
  (void)P;
  if (!dir) return MVSK_OK;
  if (part >= 2) {  // every face small: explicit face Grams, PCG rounds in shared memory
    TRY(part == 3 ? small_face_direction<kMFt>(c, bb, B) : small_face_direction<kMF>(c, bb, B));
    return batch_iteration_tail(c, bb, B, cc);
  }
  if (U) {
    TRY(hvpdiag_tc_batch_u(c, bb, B, Gz));
  } else {
    TRY(hvpdiag_tc_batch(c, bb, B, Gz));
  }
  if (K > 0)
    PROF_LAUNCH(NK_PROBE_FILL, (k_probe_fill<float><<<dim3((c->ld + 255) / 256, K, B), 256, 0, c->stream>>>(base, K)));
  PROF_LAUNCH(NK_PCG_SETUP, (k_pcg_setup<float><<<dim3(1, B), kVT, 0, c->stream>>>(base, nullptr, Gz, -1)));
  PROF_LAUNCH(NK_PCG_SETUP_COLS, (k_pcg_setup_cols<float><<<dim3(ncol1, B), 512, 0, c->stream>>>(base)));
  const unsigned gl = (unsigned)((c->ld + 255) / 256), gl4 = (unsigned)((c->ld + 1023) / 1024);
  const float invT = (float)(1.0 / (double)c->T);
  if (U)
    PROF_LAUNCH(NK_COLS, (k_cols_bf16_u<<<dim3(gl, B * ncol1), 256, 0, c->stream>>>(base, ncol1, 0, 0, bb.u_idx,
                                                                                     bb.u_info, bb.P16)));
  else
    PROF_LAUNCH(NK_COLS, (k_cols_bf16_b<<<dim3(gl4, B * ncol1), 256, 0, c->stream>>>(base, ncol1, 0, 0, bb.P16)));
  for (int it = 0; it < kmax; ++it) {
    int s2 = 0;
    KPart kp{bb.part, 0, B * ncol1, ncol1, c->ld, invT, bb.P16};
    if (U) {
      TRY(hvp_tc_batch_u(c, bb, B, ncol1, &kp.rts));
      kp.upos = bb.u_pos;
      kp.uidx = bb.u_idx;
      kp.uinfo = bb.u_info;
    } else {
      TRY(hvp_tc_batch(c, bb, B, ncol1, &s2));
      kp.splits = s2;
    }
    PROF_LAUNCH(NK_PCG_STEP, (k_pcg_step_f<<<dim3(ncol1, B), 1024, 0, c->stream>>>(base, 0, kmax, kp)));
  }
  if (K > 0) {
    TRY(U ? third_tc_batch_u(c, bb, B, K) : third_tc_batch(c, bb, B, K));
  } else {
    for (int b = 0; b < B; ++b) CU(cudaMemsetAsync(inst_at(base, b).at, 0, sizeof(double) * c->ld, c->stream));
  }
  PROF_LAUNCH(NK_PCG_SETUP2, (k_pcg_setup2<float><<<dim3(1, B), kVT, 0, c->stream>>>(base, ca, ca / 2)));
  if (U)
    PROF_LAUNCH(NK_COLS, (k_cols_bf16_u<<<dim3(gl, B), 256, 0, c->stream>>>(base, 1, ca, 0, bb.u_idx, bb.u_info,
                                                                             bb.P16)));
  else
    PROF_LAUNCH(NK_COLS, (k_cols_bf16_b<<<dim3(gl4, B), 256, 0, c->stream>>>(base, 1, ca, 0, bb.P16)));
  for (int it = 0; it < kmax; ++it) {
    int s2 = 0;
    KPart kp{bb.part, 0, B, 1, c->ld, invT, bb.P16};
    if (U) {
      TRY(hvp_tc_batch_u(c, bb, B, 1, &kp.rts));
      kp.upos = bb.u_pos;
      kp.uidx = bb.u_idx;
      kp.uinfo = bb.u_info;
    } else {
      TRY(hvp_tc_batch(c, bb, B, 1, &s2));
      kp.splits = s2;
    }
    PROF_LAUNCH(NK_PCG_STEP_A, (k_pcg_step_fc<<<dim3(kPCL, B), 512, 0, c->stream>>>(base, ca, kmax, kp)));
  }
  PROF_LAUNCH(NK_ASSEMBLE, (k_assemble<float><<<dim3(1, B), kVT, 0, c->stream>>>(base, ca)));
  return batch_iteration_tail(c, bb, B, cc);
}

// The quartic step and the boundary block of one lockstep iteration (after
// the direction block of batch_iteration).
mvsk_status batch_iteration_tail(mvsk_ctx* c, BatchBuf& bb, int B, const std::vector<std::array<double, 4>>& cc) {
  const Inst& base = bb.base;
  const bool split = c->opt.split_products != 0;
  const OzBuf& oz = c->oz;
  const int Gz = oz_row_ctas(c);
  const int Gl = split ? oz_ls_ctas(c) : c->grid;
  auto ls_split = [&](double* dvec, int skip_slot, const int* need) -> mvsk_status {
    for (int b0 = 0; b0 < B; b0 += kOzMaxB) {
      const int nb = B - b0 < kOzMaxB ? B - b0 : kOzMaxB;
      int sp = 0;
      TRY(oz_product(c, 0, dvec + (size_t)b0 * base.vs, base.vs, nb, oz_bp(nb), need, &sp));
      PROF_LAUNCH(NK_OZ_LS, (k_oz_fin_ls<<<dim3(Gl, nb), 256, 0, c->stream>>>(oz.part, sp, oz_bp(nb), oz.MpF, oz.eF,
                                                                             oz.fF, base, b0, skip_slot, bb.wls,
                                                                             nullptr, need)));
    }
    return MVSK_OK;
  };
  const bool uls = split && bb.umode && bb.u_AFU != nullptr;
  // A v on the union of the faces for B vectors v (zero off the union), gated by need (nullable)
  auto ls_union = [&](double* dvec, int skip_slot, const int* need) -> mvsk_status {
    for (int b0 = 0; b0 < B; b0 += kOzMaxB) {
      const int nb = B - b0 < kOzMaxB ? B - b0 : kOzMaxB;
      TRY(oz_product_u(c, dvec + (size_t)b0 * base.vs, base.vs, bb.u_idx, nb, oz_bp(nb), bb.u_AFU, bb.u_info, need));
      PROF_LAUNCH(NK_OZ_LS, (k_oz_fin_ls<<<dim3(Gl, nb), 256, 0, c->stream>>>(oz.part, 0, oz_bp(nb), oz.MpF, oz.eF,
                                                                             oz.fF, base, b0, skip_slot, bb.wls,
                                                                             bb.u_info, need)));
    }
    return MVSK_OK;
  };
  if (uls) {  // d is zero off the faces: A d on the union
    TRY(ls_union(base.d, SI_DONE, nullptr));
  } else if (split) {
    TRY(ls_split(base.d, SI_DONE, nullptr));
  } else {
    for (int b = 0; b < B; ++b) {
      const Inst s = inst_at(base, b);
      PassArgs a = pass_args_inst(cc[b].data());
      a.in[0] = s.d;
      a.z = s.z;
      a.skip = s.si + SI_DONE;
      TRY(run_pass(c, P64, M_LS, 1, a, nullptr, s.spart));
    }
  }
  PROF_LAUNCH(NK_DECIDE1, (k_decide1<<<dim3(1, B), kVT, 0, c->stream>>>(base, nullptr, Gl, uls ? bb.u_pos : nullptr)));
  if (split) PROF_LAUNCH(NK_ZSTEP, (k_z_step<<<dim3(Gz, B), 256, 0, c->stream>>>(base, bb.wls, 1)));
  if (split) {
    // the segment: on the union of the faces when every taken one vanishes
    // off it (checked exactly by k_decide1), else on all columns
    PROF_LAUNCH(NK_NEED, (k_need_ls2<<<1, 64, 0, c->stream>>>(base, B, bb.need, uls ? 1 : 0)));
    TRY(ls_split(base.dstep, SI_SKIPLS, bb.need));
    if (uls) TRY(ls_union(base.dstep, SI_SKIPLS, bb.need + 1));
  } else {
    for (int b = 0; b < B; ++b) {
      const Inst s = inst_at(base, b);
      PassArgs a = pass_args_inst(cc[b].data());
      a.in[0] = s.dstep;
      a.z = s.z;
      a.skip = s.si + SI_SKIPLS;
      TRY(run_pass(c, P64, M_LS, 1, a, nullptr, s.spart));
    }
  }
  PROF_LAUNCH(NK_DECIDE2, (k_decide2<<<dim3(1, B), kVT, 0, c->stream>>>(base, nullptr, Gl)));
  if (split) PROF_LAUNCH(NK_ZSTEP, (k_z_step<<<dim3(Gz, B), 256, 0, c->stream>>>(base, bb.wls, 2)));
  PROF_LAUNCH(NK_END_ITER, (k_end_iter<<<dim3(1, B), 32, 0, c->stream>>>(base)));
  return MVSK_OK;
}

// Per-instance host state: stall-recovery phases and the target calibration.
struct InstRun {
  double lam[4] = {0, 0, 0, 0}, target = NAN;
  std::array<double, 4> cc{};
  int phase = 0;
  // 0 no target, 1 lower-end solve, 2 growing, 3 Illinois, 4 first solve at
  // a point of its group's c1 grid, 5 waiting for the rest of that grid
  int cal = 0;
  double c_lo = 0, c_hi = 0, h_lo = 0, h_hi = 0, c1_ref = 0, c1_max = 0;
  int side = 0, evals = 0, iters = 0, restarts = 0;
  int run_status = MVSK_OK;
  bool finished = false, final_from_hi = false;
  std::chrono::steady_clock::time_point t_start;
  double ev[3] = {0, 0, 0};
  double kkt0 = NAN;  // kkt_rel normaliser when the result is another lane's grid point
  int last_its = -1;  // iterations of the last finished inner solve
};

// Requests of one lockstep batch that share (c2, c3, c4) and each carry a
// return target trace one curve m(c1) = mu^T x*(c1) (non-decreasing in c1).
// Their first inner solves run at the points of a c1 grid, one per request:
// c1 = 0 for the lowest target and c1_ref 2^(-6 .. 2) log-spaced for the
// others (c1_ref: the c1 at which mean and variance trade evenly), all from
// 1/n.  Every finished grid point (c1, its minimiser and z = A x*) is kept,
// and each request brackets its own target from the whole grid before the
// same Illinois iteration as a single request (or the growth x8 when the grid
// stays below its target).  The root is the one each request would reach
// alone: the calibration stops on the same tests.
struct GroupPt {
  double c1, mean, f, kkt, kkt0;
  int slot;  // lane whose pool slot holds x*(c1) and z
};
struct CalGroup {
  std::vector<GroupPt> pts;
  int pending = 0;  // grid solves not finished yet
};

// Start an inner solve of instance b at c1 from warm start w0 (device vector or
// null: 1/n).  zw0: the cached A w0 (device, T) when known; without it the next
// iteration recomputes z = A x (split products; a start from 1/n takes A 1/n).
// Start of an inner solve in lane b, one launch: the state of k_init_state
// (options h, iteration budget, probes, ...) followed by the first phase of
// k_new_phase (thread 0), x from w0 (ld values) or 1/n on the n coordinates,
// and z = A x from zs when given (T values).
struct LaneStart {
  double h[12];
  double tol, eta;
  int maxit, stallwin, probes, kmaxit, arcmax, lsrule;
  unsigned long long seed;
};
__global__ void __launch_bounds__(256) k_start_lane(Inst base, int b, LaneStart a, const double* w0,
                                                    const double* zs) {
  const Inst s = inst_at(base, b);
  const int n = s.n, ld = s.ld;
  const double inv_n = 1.0 / (double)n;
  for (int i = threadIdx.x; i < ld; i += blockDim.x) s.x[i] = w0 != nullptr ? w0[i] : (i < n ? inv_n : 0.0);
  if (zs != nullptr)
    for (long long t = threadIdx.x; t < s.T; t += blockDim.x) s.z[t] = zs[t];
  if (threadIdx.x == 0) {
    for (int q = 0; q < kSI; ++q) s.si[q] = 0;
    for (int q = SD_HIST; q < kSD; ++q) s.sd[q] = 0.0;
    s.sd[SD_TOL] = a.tol;
    s.sd[SD_BEST] = INFINITY;
    s.sd[SD_TAU] = a.h[0];
    s.sd[SD_EPSACT] = a.h[1];
    s.sd[SD_RELRATIO] = a.h[2];
    s.sd[SD_REG] = a.h[3];
    s.sd[SD_KTOL] = a.h[4];
    s.sd[SD_C1] = a.h[5];
    s.sd[SD_C2] = a.h[6];
    s.sd[SD_C3] = a.h[7];
    s.sd[SD_C4] = a.h[8];
    s.sd[SD_INVT] = a.h[9];
    s.sd[SD_DESCEPS] = a.h[10];
    s.sd[SD_STALLF] = a.h[11];
    s.si[SI_PCG] = 1;
    s.si[SI_PROBES] = a.probes;
    s.si[SI_SEEDLO] = (int)(unsigned)(a.seed & 0xffffffffull);
    s.si[SI_SEEDHI] = (int)(unsigned)(a.seed >> 32);
    s.si[SI_KMAXIT] = a.kmaxit;
    s.si[SI_ARCMAX] = a.arcmax;
    s.si[SI_LSRULE] = a.lsrule;
    // first phase (SI_DONE, SI_PHASEIT, SI_HISTN are zero from above)
    s.si[SI_MAXIT] = a.maxit;
    s.si[SI_STALLWIN] = a.stallwin;
    s.sd[SD_ETA] = a.eta;
  }
}

mvsk_status batch_start_run(mvsk_ctx* c, BatchBuf& bb, int b, InstRun& r, double c1, const double* w0, double tol,
                            const double* zw0) {
  r.cc[0] = c1;
  const Options& o = c->opt;
  const double reg = isnan(o.reg) ? 1e-4 : o.reg;
  LaneStart a{{o.tau, o.eps_act, o.release_ratio, reg, o.krylov_tol, r.cc[0], r.cc[1], r.cc[2], r.cc[3],
               1.0 / (double)c->T, o.descent_eps, o.stall_factor},
              tol, o.eta, o.pcg_max_iter, o.stall_window, o.probes, o.krylov_maxit, o.arc_halvings, o.line_search,
              o.probe_seed};
  // the KKT residual at the 1/n start (kkt_rel normaliser) of every instance
  // started in this round is evaluated by one k_kkt0_batch (kkt0_flush)
  bb.kq_idx.push_back(b);
  bb.kq_c1.push_back(c1);
  const double* zs = w0 == nullptr ? bb.z0 : zw0;
  if (zs == nullptr) bb.needz_req = 1;
  k_start_lane<<<1, 256, 0, c->stream>>>(bb.base, b, a, w0, zs);
  c->launches += 1;
  CU(cudaGetLastError());
  r.phase = 0;
  r.evals += 1;
  r.t_start = std::chrono::steady_clock::now();
  return MVSK_OK;
}

// One k_kkt0_batch for the inner solves started since the last flush.
mvsk_status kkt0_flush(mvsk_ctx* c, BatchBuf& bb) {
  const int n = (int)bb.kq_idx.size();
  if (n == 0) return MVSK_OK;
  // pageable sources: each copy has taken its data when the call returns
  double* c1d = reinterpret_cast<double*>(bb.kq_dev);
  int* idxd = reinterpret_cast<int*>(c1d + bb.cap);
  CU(cudaMemcpyAsync(c1d, bb.kq_c1.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(idxd, bb.kq_idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
  k_kkt0_batch<<<dim3(1, n), kVT, 0, c->stream>>>(bb.base, idxd, c1d, bb.G0);
  c->launches += 1;
  CU(cudaGetLastError());
  bb.kq_idx.clear();
  bb.kq_c1.clear();
  return MVSK_OK;
}

// Buffers of the face-restricted products (context lifetime; sizes depend on
// T and n only).
mvsk_status ensure_ubuf(mvsk_ctx* c, BatchBuf& bb) {
  if (bb.u_AU != nullptr) return MVSK_OK;
  void* p;
  const size_t ld = (size_t)c->ld;
  TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * (size_t)c->T * ld));
  bb.u_AU = (__nv_bfloat16*)p;
  TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * ld * (size_t)c->Tp));
  bb.u_AUT = (__nv_bfloat16*)p;
  TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * ld * (size_t)c->Tp));
  bb.u_A2UT = (__nv_bfloat16*)p;
  TRY(dalloc(c, &p, sizeof(int) * (3 * ld + 8 + 4 * kUMaxProds)));
  bb.u_flag = (int*)p;
  bb.u_idx = bb.u_flag + ld;
  bb.u_pos = bb.u_idx + ld;
  bb.u_info = bb.u_pos + ld;
  bb.u_rt = bb.u_info + 8;
  TRY(dalloc(c, &p, sizeof(UProd) * kUMaxProds));
  bb.u_specs = (UProd*)p;
  CU(cudaMemsetAsync(bb.u_AU, 0, sizeof(__nv_bfloat16) * (size_t)c->T * ld, c->stream));
  CU(cudaMemsetAsync(bb.u_AUT, 0, sizeof(__nv_bfloat16) * ld * (size_t)c->Tp, c->stream));
  CU(cudaMemsetAsync(bb.u_A2UT, 0, sizeof(__nv_bfloat16) * ld * (size_t)c->Tp, c->stream));
  CU(cudaMemsetAsync(bb.u_specs, 0, sizeof(UProd) * kUMaxProds, c->stream));
  if (c->opt.split_products) {  // the line-search product on U
    TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * kOzS * (size_t)c->oz.MpF * ld));
    bb.u_AFU = (__nv_bfloat16*)p;
  }
  CU(cudaFuncSetAttribute(k_pcg_round_small<kMF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)(sizeof(float) * face_gram_words<kMF>())));
  CU(cudaFuncSetAttribute(k_pcg_round_small<kMFt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)(sizeof(float) * face_gram_words<kMFt>())));
  CU(cudaFuncSetAttribute(k_face_hutch<kMF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)HutchTc<kMF>::kSmem));
  CU(cudaFuncSetAttribute(k_face_hutch<kMFt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)HutchTc<kMFt>::kSmem));
  CU(cudaFuncSetAttribute(k_face_gram_tc<kMF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GramTc<kMF>::kSmem));
  CU(cudaFuncSetAttribute(k_face_gram_tc<kMFt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)GramTc<kMFt>::kSmem));
  return MVSK_OK;
}

// Iterations between full recomputations of the cached z = A x of a batch.
constexpr int kZRefresh = 32;

mvsk_status batch_solve(mvsk_ctx* c, int B, const double* lam_h, const double* tg_h, double tol, const double* W0,
                        double* W_out, mvsk_info* infos) {
  BatchBuf& bb = c->batch;
  const Options& o = c->opt;
  // Lanes: instances advanced together by the lockstep graph.  With
  // batch_lanes = L < B (split products only) the B requests queue for L lanes
  // and a lane whose request has finished takes the next one (continuous
  // batching): the graph reads every per-instance parameter on the device.
  const bool split = o.split_products != 0;
  const int L = (split && o.batch_lanes > 0 && o.batch_lanes < B) ? o.batch_lanes : B;
  TRY(ensure_tc_pcg(c));
  TRY(batch_alloc(c, bb, L));
  const auto t0 = std::chrono::steady_clock::now();
  const double s_eq = c->s_equal;
  const bool stdz = o.pref_scaling == 1 && s_eq > 0.0 && isfinite(s_eq);
  const double scale = c->mu_absmax, gap_tol = o.cal_rel_tol * scale;
  const size_t ld = (size_t)c->ld;
  // per-request data
  std::vector<InstRun> req((size_t)B);
  std::vector<std::array<double, 4>> ccq((size_t)B);
  for (int q = 0; q < B; ++q) {
    InstRun& r = req[(size_t)q];
    for (int k = 0; k < 4; ++k) {
      r.lam[k] = lam_h[4 * q + k];
      r.cc[k] = stdz ? r.lam[k] / pow(s_eq, k + 1) : r.lam[k];
    }
    r.target = tg_h[q];
    ccq[(size_t)q] = r.cc;
    r.c1_ref = fmax(r.cc[1], 1e-300) * s_eq * s_eq / fmax(scale, 1e-300);
    r.c1_max = 1e6 * r.c1_ref;
  }
  std::vector<InstRun> run((size_t)L);
  std::vector<int> lane_req((size_t)L, -1);
  bb.needz_req = 0;
  std::vector<std::array<double, 4>> cc(ccq.begin(), ccq.begin() + L);
  // device buffers for warm starts: instance scratch columns 20 (lo) and 21 (hi)
  auto xlo = [&](int b) { return inst_at(bb.base, b).tmp + (size_t)20 * ld; };
  auto xhi = [&](int b) { return inst_at(bb.base, b).tmp + (size_t)21 * ld; };
  // their cached z = A x (split products)
  auto zlo = [&](int b) { return bb.zsave + (size_t)(2 * b) * c->T; };
  auto zhi = [&](int b) { return bb.zsave + (size_t)(2 * b + 1) * c->T; };
  auto save_z = [&](double* dst, const double* src) -> mvsk_status {
    if (split) CU(cudaMemcpyAsync(dst, src, sizeof(double) * c->T, cudaMemcpyDeviceToDevice, c->stream));
    return MVSK_OK;
  };
  std::vector<double> hw;  // validated warm starts (host), B x n
  if (W0 != nullptr) {
    hw.resize((size_t)B * c->n);
    CU(cudaMemcpy(hw.data(), W0, sizeof(double) * hw.size(), cudaMemcpyDefault));
    for (int q = 0; q < B; ++q) {
      double sm = 0.0, mn = INFINITY;
      for (int i = 0; i < c->n; ++i) {
        sm += hw[(size_t)q * c->n + i];
        mn = fmin(mn, hw[(size_t)q * c->n + i]);
      }
      if (!(fabs(sm - 1.0) <= 1e-9) || mn < o.tau * (1.0 - 1e-9)) return fail(MVSK_EINVAL, "W0 row %d not in Delta(tau)", q);
    }
  }
  if (split)  // digit planes of A are built outside the capture
    for (int b0 = 0; b0 < L; b0 += kOzMaxB) TRY(oz_prepare(c, oz_bp(L - b0 < kOzMaxB ? L - b0 : kOzMaxB)));
  // face-restricted direction products: gathered operands and index lists
  bb.umode = o.face_products != 0;
  if (bb.umode) {
    TRY(ensure_ubuf(c, bb));
    const int widths[2] = {o.probes + 1, 1};
    TRY(u_prepare(c, bb, L, widths, 2, o.probes));
  }
  c->prof_uinfo = bb.umode ? bb.u_info : nullptr;
  // graphs of one lockstep iteration (c1 is read on the device, so calibration
  // needs no re-capture): the whole iteration, or with face-restricted
  // products the oracle block (part 0) and the two direction forms (parts 1, 2)
  struct ItGraph {
    cudaGraphExec_t e = nullptr;
    cudaGraph_t g = nullptr;  // the captured graph (a child of the one-graph iteration)
    long long launches = 0;
    size_t ev_b = 0, ev_e = 0;
    ~ItGraph() {
      if (e) cudaGraphExecDestroy(e);
      if (g) cudaGraphDestroy(g);
    }
  };
  ItGraph gfull, ghead, glarge, gsmall, gnarrow, giter;
  auto capture = [&](int part, ItGraph& gr) -> mvsk_status {
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const long long l0 = c->launches;
    gr.ev_b = c->ev_kind.size();
    const mvsk_status cs = batch_iteration(c, bb, L, cc, part);
    gr.ev_e = c->ev_kind.size();
    gr.launches = c->launches - l0;
    c->launches = l0;
    const cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
    if (cs != MVSK_OK) {
      if (g) cudaGraphDestroy(g);
      return cs;
    }
    CU(ce);
    {  // a replay launches exactly the graph's kernel nodes
      size_t nn = 0;
      CU(cudaGraphGetNodes(g, nullptr, &nn));
      std::vector<cudaGraphNode_t> nodes(nn);
      CU(cudaGraphGetNodes(g, nodes.data(), &nn));
      long long nk = 0;
      for (size_t q = 0; q < nn; ++q) {
        cudaGraphNodeType t;
        CU(cudaGraphNodeGetType(nodes[q], &t));
        nk += t == cudaGraphNodeTypeKernel;
      }
      gr.launches = nk;
    }
    gr.g = g;
    CU(cudaGraphInstantiate(&gr.e, g, 0));
    return MVSK_OK;
  };
  // With face-restricted products the iteration is one graph when the
  // direction bodies hold no profiler events (conditional bodies take kernels,
  // copies and child graphs only): the oracle block, then a switch node over
  // the three direction forms on the value k_small_mode sets on the device,
  // so that no host round trip separates them.  Otherwise the host reads the
  // form after the oracle block and replays its graph.
  bool one_graph = false;
  if (bb.umode) {
    TRY(capture(1, glarge));
    TRY(capture(2, gsmall));
    TRY(capture(3, gnarrow));
    one_graph = o.face_small != 0 && glarge.ev_e == glarge.ev_b && gsmall.ev_e == gsmall.ev_b &&
                gnarrow.ev_e == gnarrow.ev_b;
    if (one_graph) {
      CU(cudaGraphCreate(&giter.g, 0));
      if (cudaGraphConditionalHandleCreate(&bb.cond, giter.g, 0, 0) != cudaSuccess) {
        cudaGetLastError();
        one_graph = false;
      }
    }
    bb.has_cond = one_graph ? 1 : 0;  // captured into k_small_mode's arguments
    const mvsk_status hs = capture(0, ghead);
    bb.has_cond = 0;
    TRY(hs);
    if (one_graph) {
      cudaGraphNode_t nh = nullptr, nc = nullptr;
      CU(cudaGraphAddChildGraphNode(&nh, giter.g, nullptr, 0, ghead.g));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = bb.cond;
      cp.conditional.type = cudaGraphCondTypeSwitch;
      cp.conditional.size = 3;  // body f runs for the form f: 0 large faces, 1 wide, 2 narrow small faces
      CU(cudaGraphAddNode(&nc, giter.g, &nh, nullptr, 1, &cp));
      const ItGraph* body[3] = {&glarge, &gsmall, &gnarrow};
      for (int q = 0; q < 3; ++q) {
        cudaGraphNode_t nb = nullptr;
        CU(cudaGraphAddChildGraphNode(&nb, cp.conditional.phGraph_out[q], nullptr, 0, body[q]->g));
      }
      CU(cudaGraphInstantiate(&giter.e, giter.g, 0));
      giter.launches = ghead.launches;  // plus the body's, counted once the form is read back
      giter.ev_b = ghead.ev_b;
      giter.ev_e = ghead.ev_e;
    }
  } else {
    TRY(capture(-1, gfull));
  }
  // A replay queues no wait: the profiled event pairs of the iteration's
  // graphs are read after the iteration's state copy (one wait per iteration).
  std::vector<const ItGraph*> pend;
  auto replay = [&](ItGraph& gr) -> mvsk_status {
    CU(cudaGraphLaunch(gr.e, c->stream));
    c->launches += gr.launches;
    if (c->prof_on) pend.push_back(&gr);
    return MVSK_OK;
  };
  auto collect = [&]() -> mvsk_status {  // after a wait that followed the replays
    const int* uinfo = c->prof_uinfo != nullptr ? c->hword + 2 : nullptr;  // copied with the state
    for (const ItGraph* g : pend) TRY(prof_collect(c, g->ev_b, g->ev_e, uinfo));
    pend.clear();
    return MVSK_OK;
  };
  int small_dir = 0;  // host copy of the direction form chosen on the device
  // c1-free part of the gradient at 1/n, once per request (psi_q depends on c2..c4 only):
  // in the lanes' G0 when every request has its lane, else per request in bb.Gq
  double* G0q = bb.G0;
  if (L < B) {
    if (bb.qcap < B) {
      if (bb.Gq != nullptr) cudaFree(bb.Gq);
      bb.Gq = nullptr;
      bb.qcap = 0;
      if (cudaMalloc(&bb.Gq, sizeof(double) * ld * (size_t)B) != cudaSuccess) {
        cudaGetLastError();
        return fail(MVSK_ENOMEM, "request buffer allocation failed");
      }
      bb.qcap = B;
    }
    G0q = bb.Gq;
  }
  if (split) {
    // z0 = A 1/n is shared: one FP64 pass, then psi'_q(z0) for the requests of
    // each group of L and one split product A^T W per 64 of them
    const Inst s0 = inst_at(bb.base, 0);
    k_fill<<<(c->ld + 255) / 256, 256, 0, c->stream>>>(s0.x, c->n, c->ld, 1.0 / c->n);
    TRY(pass_fwd_z(c, s0.x, s0.z));
    CU(cudaMemcpyAsync(bb.z0, s0.z, sizeof(double) * c->T, cudaMemcpyDeviceToDevice, c->stream));
    c->launches += 1;
    for (int q0 = 0; q0 < B; q0 += L) {
      const int nq = B - q0 < L ? B - q0 : L;
      for (int j = 0; j < nq; ++j)
        k_dpsi_into<<<(unsigned)((c->T + 255) / 256), 256, 0, c->stream>>>(
            s0.z, c->T, ccq[(size_t)(q0 + j)][1], ccq[(size_t)(q0 + j)][2], ccq[(size_t)(q0 + j)][3],
            bb.Wt + (size_t)j * c->T);
      c->launches += nq;
      CU(cudaGetLastError());
      for (int b0 = 0; b0 < nq; b0 += kOzMaxB) {
        const int nb = nq - b0 < kOzMaxB ? nq - b0 : kOzMaxB;
        int sp = 0;
        TRY(oz_product(c, 1, bb.Wt + (size_t)b0 * c->T, c->T, nb, oz_bp(nb), nullptr, &sp));
        k_oz_store<<<dim3((unsigned)((c->n + 255) / 256), (unsigned)nb), 256, 0, c->stream>>>(
            c->oz.part, sp, oz_bp(nb), c->oz.MpB, c->n, nb, c->oz.eB, c->oz.fB, 1.0 / (double)c->T,
            G0q + (size_t)(q0 + b0) * c->ld, c->ld);
        c->launches += 1;
        CU(cudaGetLastError());
      }
    }
  } else {
    for (int b = 0; b < B; ++b) {
      const Inst s = inst_at(bb.base, b);
      k_fill<<<(c->ld + 255) / 256, 256, 0, c->stream>>>(s.x, c->n, c->ld, 1.0 / c->n);
      PassArgs a = pass_args_inst(cc[(size_t)b].data());
      a.in[0] = s.x;
      a.rowout = s.z;
      TRY(run_pass(c, P64, M_VALGRAD, 1, a, nullptr, s.spart));
      TRY(reduce_cols(c, P64, 1, bb.G0 + (size_t)b * c->ld, c->ld, nullptr, 0.0, nullptr, nullptr));
      c->launches += 1;
    }
  }
  // user warm starts on the device (Wq, ld-strided) with their z = A w0 (Zq, one
  // split product per 64 requests), so that a lane taking such a request needs
  // no recomputation of z for the whole batch
  if (!hw.empty()) {
    if (bb.wcap < B) {
      if (bb.Wq != nullptr) cudaFree(bb.Wq);
      if (bb.Zq != nullptr) cudaFree(bb.Zq);
      bb.Wq = bb.Zq = nullptr;
      bb.wcap = 0;
      if (cudaMalloc(&bb.Wq, sizeof(double) * ld * (size_t)B) != cudaSuccess ||
          cudaMalloc(&bb.Zq, sizeof(double) * (size_t)c->T * (size_t)B) != cudaSuccess) {
        cudaGetLastError();
        return fail(MVSK_ENOMEM, "warm-start buffer allocation failed");
      }
      bb.wcap = B;
    }
    CU(cudaMemsetAsync(bb.Wq, 0, sizeof(double) * ld * (size_t)B, c->stream));
    CU(cudaMemcpy2DAsync(bb.Wq, sizeof(double) * ld, hw.data(), sizeof(double) * c->n, sizeof(double) * c->n,
                         (size_t)B, cudaMemcpyHostToDevice, c->stream));
    if (split) {
      for (int q0 = 0; q0 < B; q0 += kOzMaxB) {
        const int nb = B - q0 < kOzMaxB ? B - q0 : kOzMaxB;
        int sp = 0;
        TRY(oz_product(c, 0, bb.Wq + (size_t)q0 * ld, c->ld, nb, oz_bp(nb), nullptr, &sp));
        k_oz_store<<<dim3((unsigned)((c->T + 255) / 256), (unsigned)nb), 256, 0, c->stream>>>(
            c->oz.part, sp, oz_bp(nb), c->oz.MpF, c->T, nb, c->oz.eF, c->oz.fF, 1.0, bb.Zq + (size_t)q0 * c->T,
            c->T);
        c->launches += 1;
        CU(cudaGetLastError());
      }
    }
  }
  // Calibration groups (see CalGroup): every request has its own lane and no
  // user warm start, with split products (the grid points keep their cached z).
  std::vector<int> group_of((size_t)B, -1);
  std::vector<double> grid_c1((size_t)B, 0.0);
  std::vector<CalGroup> groups;
  if (o.group_cal && split && L == B && hw.empty()) {
    std::vector<int> idx;
    for (int q = 0; q < B; ++q)
      if (!isnan(req[(size_t)q].target)) idx.push_back(q);
    std::vector<char> used((size_t)B, 0);
    for (int q : idx) {
      if (used[(size_t)q]) continue;
      std::vector<int> mem;
      for (int p2 : idx)
        if (!used[(size_t)p2] && ccq[(size_t)p2][1] == ccq[(size_t)q][1] && ccq[(size_t)p2][2] == ccq[(size_t)q][2] &&
            ccq[(size_t)p2][3] == ccq[(size_t)q][3]) {
          mem.push_back(p2);
          used[(size_t)p2] = 1;
        }
      if (mem.size() < 2) continue;
      std::stable_sort(mem.begin(), mem.end(),
                       [&](int a, int b2) { return req[(size_t)a].target < req[(size_t)b2].target; });
      const int G = (int)mem.size();
      for (int k = 0; k < G; ++k) {
        group_of[(size_t)mem[(size_t)k]] = (int)groups.size();
        const double e = G == 2 ? 0.0 : -6.0 + 8.0 * (double)(k - 1) / (double)(G - 2);
        grid_c1[(size_t)mem[(size_t)k]] = k == 0 ? 0.0 : req[(size_t)mem[(size_t)k]].c1_ref * exp2(e);
      }
      CalGroup g;
      g.pending = G;
      groups.push_back(g);
    }
    if (!groups.empty() && bb.gcap < B) {
      if (bb.gpool != nullptr) cudaFree(bb.gpool);
      bb.gpool = nullptr;
      bb.gcap = 0;
      if (cudaMalloc(&bb.gpool, sizeof(double) * (ld + (size_t)c->T) * (size_t)B) != cudaSuccess) {
        cudaGetLastError();
        return fail(MVSK_ENOMEM, "calibration grid buffer allocation failed");
      }
      bb.gcap = B;
    }
  }
  // pool slot of lane b: a grid point's x* (ld) and its cached z (T)
  auto gx = [&](int b) { return bb.gpool + (size_t)b * (ld + (size_t)c->T); };
  auto gz = [&](int b) { return gx(b) + ld; };
  // request q into lane b: its state, its G0 and warm start, and the first inner solve
  int next_req = 0;
  auto assign = [&](int b) -> mvsk_status {
    const int q = next_req++;
    lane_req[(size_t)b] = q;
    run[(size_t)b] = req[(size_t)q];
    InstRun& r = run[(size_t)b];
    const Inst s = inst_at(bb.base, b);
    if (G0q != bb.G0)
      CU(cudaMemcpyAsync(bb.G0 + (size_t)b * ld, G0q + (size_t)q * ld, sizeof(double) * ld, cudaMemcpyDeviceToDevice,
                         c->stream));
    const double* w0 = nullptr;
    if (!hw.empty()) {
      CU(cudaMemcpyAsync(s.xbar, bb.Wq + (size_t)q * ld, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
      w0 = s.xbar;
    }
    if (isnan(r.target)) {
      r.cal = 0;
      return batch_start_run(c, bb, b, r, r.cc[0], w0, tol,
                             (w0 != nullptr && split) ? bb.Zq + (size_t)q * c->T : nullptr);
    }
    if (group_of[(size_t)q] >= 0) {
      r.cal = 4;
      return batch_start_run(c, bb, b, r, grid_c1[(size_t)q], nullptr, tol, nullptr);
    }
    r.cal = 1;
    return batch_start_run(c, bb, b, r, 0.0, nullptr, tol, nullptr);
  };
  // results of the request in lane b (at the end of its last inner solve):
  // W out, and the request's counters and evaluations copied into pinned
  // per-request slots that the infos read after the final wait (no wait here)
  if (infos != nullptr && bb.qhcap < B) {
    if (bb.q_si != nullptr) cudaFreeHost(bb.q_si);
    if (bb.q_ev != nullptr) cudaFreeHost(bb.q_ev);
    bb.q_si = nullptr;
    bb.q_ev = nullptr;
    bb.qhcap = 0;
    if (cudaMallocHost(&bb.q_si, sizeof(int) * kSI * (size_t)B) != cudaSuccess ||
        cudaMallocHost(&bb.q_ev, sizeof(double) * 4 * (size_t)B) != cudaSuccess) {
      cudaGetLastError();
      return fail(MVSK_ENOMEM, "pinned request slot allocation failed");
    }
    bb.qhcap = B;
  }
  mvsk_status first = MVSK_OK;
  auto emit = [&](int b) -> mvsk_status {
    InstRun& r = run[(size_t)b];
    const int q = lane_req[(size_t)b];
    const Inst s = inst_at(bb.base, b);
    double* qe = infos != nullptr ? bb.q_ev + 4 * (size_t)q : nullptr;
    if (r.final_from_hi) {  // re-evaluate at the bracket end that is returned
      PassArgs a = pass_args_inst(r.cc.data());
      double c1 = r.cc[0];
      CU(cudaMemcpyAsync(s.sd + SD_C1, &c1, sizeof(double), cudaMemcpyHostToDevice, c->stream));
      a.in[0] = s.x;
      a.rowout = s.z;
      TRY(run_pass(c, P64, M_VALGRAD, 1, a, nullptr, s.spart));
      TRY(reduce_cols(c, P64, 1, s.g, c->ld, c->mu, 0.0, nullptr, nullptr, s.sd + SD_C1));
      k_eval_finish<<<1, kVT, 0, c->stream>>>(s, nullptr, c->grid, s.tmp + (size_t)23 * ld);
      c->launches += 1;
      if (qe != nullptr)
        CU(cudaMemcpyAsync(qe, s.tmp + (size_t)23 * ld, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    } else if (qe != nullptr) {
      for (int k = 0; k < 3; ++k) qe[k] = r.ev[k];
    }
    CU(cudaMemcpyAsync(W_out + (size_t)q * c->n, s.x, sizeof(double) * c->n, cudaMemcpyDefault, c->stream));
    if (infos != nullptr) {
      if (isnan(r.kkt0)) CU(cudaMemcpyAsync(qe + 3, s.sd + SD_KKT0, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      else qe[3] = r.kkt0;
      CU(cudaMemcpyAsync(bb.q_si + (size_t)q * kSI, s.si, sizeof(int) * kSI, cudaMemcpyDeviceToHost, c->stream));
      mvsk_info& inf = infos[q];
      memset(&inf, 0, sizeof(inf));
      inf.iters = r.iters;
      inf.restarts = r.restarts;
      inf.evals = r.evals;
      for (int k = 0; k < 4; ++k) inf.c[k] = r.cc[k];
      inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      inf.status = r.run_status;
    }
    if (r.run_status != MVSK_OK && first == MVSK_OK) first = (mvsk_status)r.run_status;
    return MVSK_OK;
  };
  // start the first L requests
  for (int b = 0; b < L; ++b) TRY(assign(b));
  TRY(kkt0_flush(c, bb));
  if (bb.hcap < L) {  // pinned, so that the per-iteration copies are asynchronous
    if (bb.si_h != nullptr) cudaFreeHost(bb.si_h);
    if (bb.sd_h != nullptr) cudaFreeHost(bb.sd_h);
    if (bb.ev_h != nullptr) cudaFreeHost(bb.ev_h);
    bb.si_h = nullptr;
    bb.sd_h = nullptr;
    bb.ev_h = nullptr;
    bb.hcap = 0;
    if (cudaMallocHost(&bb.si_h, sizeof(int) * kSI * (size_t)L) != cudaSuccess ||
        cudaMallocHost(&bb.sd_h, sizeof(double) * kSD * (size_t)L) != cudaSuccess ||
        cudaMallocHost(&bb.ev_h, sizeof(double) * 4 * (size_t)L) != cudaSuccess) {
      cudaGetLastError();
      return fail(MVSK_ENOMEM, "pinned host state allocation failed");
    }
    bb.hcap = L;
  }
  int* const si = bb.si_h;
  const double* const sdh = bb.sd_h;
  double* const evh = bb.ev_h;
  const double phase_eta[3] = {o.eta, o.restart_eta1, o.restart_eta2};
  const int phase_it[3] = {o.pcg_max_iter, o.restart_iter1, o.restart_iter2};
  int remaining = B;
  long long guard_iters = 0;
  int needz_dev = 0;  // value of bb.needz on the device (a previous solve may have left 1)
  if (split) CU(cudaMemsetAsync(bb.needz, 0, sizeof(int), c->stream));
  while (remaining > 0) {
    if (split) {  // z = A x recomputed for user warm starts and every kZRefresh iterations (bounds the drift)
      const int want = (bb.needz_req || (guard_iters > 0 && guard_iters % kZRefresh == 0)) ? 1 : 0;
      if (want != needz_dev) {
        CU(cudaMemcpyAsync(bb.needz, &want, sizeof(int), cudaMemcpyHostToDevice, c->stream));
        needz_dev = want;
      }
      bb.needz_req = 0;
    }
    if (one_graph) {  // oracle block and the direction form it chose, one replay
      TRY(replay(giter));
      CU(cudaMemcpyAsync(c->hword + 1, bb.u_info + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    } else if (bb.umode) {  // oracle block, then the direction form every face allows
      TRY(replay(ghead));
      small_dir = 0;
      if (o.face_small) {
        CU(cudaMemcpyAsync(c->hword + 1, bb.u_info + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        TRY(sync(c));
        small_dir = c->hword[1];
      }
      TRY(replay(small_dir == 2 ? gnarrow : (small_dir == 1 ? gsmall : glarge)));
    } else {
      TRY(replay(gfull));
    }
    guard_iters += 1;
    // the lanes' integer and scalar states (an inner solve that converged is
    // evaluated from them: f, KKT residual, mu^T x and its kkt0 normaliser)
    CU(cudaMemcpyAsync(si, bb.base.si, sizeof(int) * kSI * (size_t)L, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(bb.sd_h, bb.base.sd, sizeof(double) * kSD * (size_t)L, cudaMemcpyDeviceToHost, c->stream));
    if (c->prof_on && c->prof_uinfo != nullptr)
      CU(cudaMemcpyAsync(c->hword + 2, c->prof_uinfo, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    TRY(sync(c));
    TRY(collect());
    if (one_graph) {
      const int f = c->hword[1];
      c->launches += (f == 2 ? gnarrow : (f == 1 ? gsmall : glarge)).launches;
    }
    // finished inner solves (host checks after every iteration): evaluate them together
    std::vector<int> fin;
    for (int b = 0; b < L; ++b) {
      InstRun& r = run[(size_t)b];
      if (lane_req[(size_t)b] < 0 || r.finished || r.cal == 5) continue;
      const int done = si[(size_t)b * kSI + SI_DONE];
      if (done == 0) {
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - r.t_start).count();
        if (el > o.max_elapsed) {  // out of time: stop this inner solve here
          const int four = 4;
          CU(cudaMemcpyAsync(inst_at(bb.base, b).si + SI_DONE, &four, sizeof(int), cudaMemcpyHostToDevice, c->stream));
          TRY(sync(c));
          si[(size_t)b * kSI + SI_DONE] = 4;
        } else {
          continue;
        }
      }
      const int d2 = si[(size_t)b * kSI + SI_DONE];
      if (d2 == 2 && r.phase + 1 < 3) {
        r.phase += 1;
        r.restarts += 1;
        k_new_phase<<<1, 32, 0, c->stream>>>(inst_at(bb.base, b), phase_eta[r.phase], phase_it[r.phase],
                                             r.phase + 1 < 3 ? o.stall_window : 0);
        c->launches += 1;
        CU(cudaGetLastError());
        continue;
      }
      r.run_status = d2 == 1 ? MVSK_OK : (d2 == 3 ? MVSK_ENUMERIC : (d2 == 4 ? MVSK_ETIMEOUT : MVSK_ENOTCONVERGED));
      r.iters += si[(size_t)b * kSI + SI_ITER];
      r.last_its = si[(size_t)b * kSI + SI_ITER];
      const Inst s = inst_at(bb.base, b);
      if (r.run_status != MVSK_OK) CU(cudaMemcpyAsync(s.x, s.bestx, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
      fin.push_back(b);
    }
    if (fin.empty()) continue;
    bool restored = false;
    for (int b : fin) {
      const Inst s = inst_at(bb.base, b);
      const double* sdb = sdh + (size_t)b * kSD;
      evh[4 * (size_t)b + 3] = sdb[SD_KKT0];
      if (run[(size_t)b].run_status == MVSK_OK) {  // the oracle block that declared convergence evaluated x
        evh[4 * (size_t)b] = sdb[SD_F];
        evh[4 * (size_t)b + 1] = sdb[SD_KKT];
        evh[4 * (size_t)b + 2] = sdb[SD_MUX];
      } else {  // the best iterate was restored: evaluate it
        PassArgs a = pass_args_inst(run[(size_t)b].cc.data());
        a.in[0] = s.x;
        a.rowout = s.z;
        TRY(run_pass(c, P64, M_VALGRAD, 1, a, nullptr, s.spart));
        TRY(reduce_cols(c, P64, 1, s.g, c->ld, c->mu, 0.0, nullptr, nullptr, s.sd + SD_C1));
        k_eval_finish<<<1, kVT, 0, c->stream>>>(s, nullptr, c->grid, s.tmp + (size_t)23 * ld);
        CU(cudaMemcpyAsync(evh + 4 * (size_t)b, s.tmp + (size_t)23 * ld, 3 * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
        c->launches += 1;
        restored = true;
      }
    }
    if (restored) TRY(sync(c));
    std::vector<int> freed;
    auto finish_b = [&](int b, bool from_hi) -> mvsk_status {
      InstRun& r = run[(size_t)b];
      if (from_hi) {
        CU(cudaMemcpyAsync(inst_at(bb.base, b).x, xhi(b), sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
        r.cc[0] = r.c_hi;
        r.final_from_hi = true;
      }
      r.finished = true;
      remaining -= 1;
      freed.push_back(b);
      return MVSK_OK;
    };
    auto illinois_b = [&](int b) -> mvsk_status {
      InstRun& r = run[(size_t)b];
      if (r.evals >= o.cal_max_evals) return finish_b(b, true);
      double cm = r.c_hi - r.h_hi * (r.c_hi - r.c_lo) / (r.h_hi - r.h_lo);
      if (!(r.c_lo < cm && cm < r.c_hi)) cm = 0.5 * (r.c_lo + r.c_hi);
      const bool lo = (cm - r.c_lo) <= (r.c_hi - cm);
      r.cal = 3;
      return batch_start_run(c, bb, b, r, cm, lo ? xlo(b) : xhi(b), tol, split ? (lo ? zlo(b) : zhi(b)) : nullptr);
    };
    // A grid request's next step from every finished point of its group: the
    // result itself when a point meets the target (c1 = 0 when its mean is
    // already high enough), else the tightest bracket for Illinois, else the
    // growth from the highest point once the grid is complete; it waits while
    // points that could bracket it are still running.
    auto group_decide = [&](int b) -> mvsk_status {
      InstRun& r = run[(size_t)b];
      const CalGroup& G = groups[(size_t)group_of[(size_t)lane_req[(size_t)b]]];
      const GroupPt *lo = nullptr, *hi = nullptr, *hit = nullptr, *zero = nullptr;
      for (const GroupPt& p : G.pts) {
        const double hp = p.mean - r.target;
        if (p.c1 == 0.0) zero = &p;
        if (fabs(hp) <= gap_tol && (hit == nullptr || fabs(hp) < fabs(hit->mean - r.target))) hit = &p;
        if (hp < 0.0) {
          if (lo == nullptr || p.c1 > lo->c1) lo = &p;
        } else if (hi == nullptr || p.c1 < hi->c1) {
          hi = &p;
        }
      }
      const Inst s = inst_at(bb.base, b);
      auto take = [&](const GroupPt& p) -> mvsk_status {  // p is this request's result
        if (p.slot != b)
          CU(cudaMemcpyAsync(s.x, gx(p.slot), sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
        r.cc[0] = p.c1;
        r.ev[0] = p.f;
        r.ev[1] = p.kkt;
        r.ev[2] = p.mean;
        r.kkt0 = p.kkt0;
        return finish_b(b, false);
      };
      auto keep = [&](const GroupPt& p, double* xd, double* zd) -> mvsk_status {
        CU(cudaMemcpyAsync(xd, gx(p.slot), sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
        CU(cudaMemcpyAsync(zd, gz(p.slot), sizeof(double) * c->T, cudaMemcpyDeviceToDevice, c->stream));
        return MVSK_OK;
      };
      if (zero != nullptr && zero->mean - r.target >= -gap_tol) return take(*zero);
      if (hit != nullptr) return take(*hit);
      if (lo != nullptr && hi != nullptr) {
        r.c_lo = lo->c1;
        r.h_lo = lo->mean - r.target;
        r.c_hi = hi->c1;
        r.h_hi = hi->mean - r.target;
        TRY(keep(*lo, xlo(b), zlo(b)));
        TRY(keep(*hi, xhi(b), zhi(b)));
        if (r.c_hi - r.c_lo <= o.cal_bracket_tol * r.c_hi) return take(*hi);
        r.side = 0;
        return illinois_b(b);
      }
      if (G.pending > 0) {  // the rest of the grid may still bracket the target
        r.cal = 5;
        return MVSK_OK;
      }
      if (lo == nullptr) {  // no point below the target (c1 = 0 did not finish): the single-request path
        r.cal = 1;
        return batch_start_run(c, bb, b, r, 0.0, nullptr, tol, nullptr);
      }
      if (lo->c1 >= r.c1_max) return take(*lo);
      r.c_lo = lo->c1;
      r.h_lo = lo->mean - r.target;
      TRY(keep(*lo, xlo(b), zlo(b)));
      r.c_hi = lo->c1 > 0.0 ? fmin(8.0 * lo->c1, r.c1_max) : (r.lam[0] > 0.0 ? (stdz ? r.lam[0] / s_eq : r.lam[0]) : r.c1_ref);
      r.cal = 2;
      return batch_start_run(c, bb, b, r, r.c_hi, xlo(b), tol, zlo(b));
    };
    for (int b : fin) {
      InstRun& r = run[(size_t)b];
      const Inst s = inst_at(bb.base, b);
      for (int q = 0; q < 3; ++q) r.ev[q] = evh[4 * (size_t)b + q];
      const double h = r.ev[2] - r.target;
      auto finish = [&](bool from_hi) -> mvsk_status { return finish_b(b, from_hi); };
      auto illinois = [&]() -> mvsk_status { return illinois_b(b); };
      if (r.cal == 4) {  // a grid point: into the group's pool, then the request's next step
        CalGroup& G = groups[(size_t)group_of[(size_t)lane_req[(size_t)b]]];
        CU(cudaMemcpyAsync(gx(b), s.x, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
        CU(cudaMemcpyAsync(gz(b), s.z, sizeof(double) * c->T, cudaMemcpyDeviceToDevice, c->stream));
        G.pts.push_back({r.cc[0], r.ev[2], r.ev[0], r.ev[1], evh[4 * (size_t)b + 3], b});
        G.pending -= 1;
        r.cal = 5;
        continue;  // decided below, with every point of this round in the pool
      }
      if (r.cal == 0) {
        TRY(finish(false));
      } else if (r.cal == 1) {
        if (h >= -gap_tol) {
          TRY(finish(false));
        } else {
          CU(cudaMemcpyAsync(xlo(b), s.x, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
          TRY(save_z(zlo(b), s.z));
          r.c_lo = 0.0;
          r.h_lo = h;
          r.c_hi = r.lam[0] > 0.0 ? (stdz ? r.lam[0] / s_eq : r.lam[0]) : r.c1_ref;
          r.cal = 2;
          TRY(batch_start_run(c, bb, b, r, r.c_hi, xlo(b), tol, split ? zlo(b) : nullptr));
        }
      } else if (r.cal == 2) {
        r.h_hi = h;
        CU(cudaMemcpyAsync(xhi(b), s.x, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
        TRY(save_z(zhi(b), s.z));
        if (h < 0.0 && r.c_hi < r.c1_max) {
          r.c_lo = r.c_hi;
          r.h_lo = r.h_hi;
          CU(cudaMemcpyAsync(xlo(b), xhi(b), sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
          TRY(save_z(zlo(b), zhi(b)));
          r.c_hi = fmin(8.0 * r.c_hi, r.c1_max);
          TRY(batch_start_run(c, bb, b, r, r.c_hi, xlo(b), tol, split ? zlo(b) : nullptr));
        } else if (h < 0.0 || fabs(h) <= gap_tol) {
          TRY(finish(false));
        } else {
          r.side = 0;
          TRY(illinois());
        }
      } else {
        const double cm = r.cc[0];
        // a solve that needed no iteration from its warm start resolves the
        // mean no finer: its point ends the calibration near the target
        if (fabs(h) <= gap_tol || (r.last_its == 0 && fabs(h) <= 10.0 * gap_tol) ||
            (r.c_hi - r.c_lo) <= o.cal_bracket_tol * r.c_hi) {
          TRY(finish(false));
        } else {
          if (h < 0.0) {
            r.c_lo = cm;
            r.h_lo = h;
            CU(cudaMemcpyAsync(xlo(b), s.x, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
            TRY(save_z(zlo(b), s.z));
            if (r.side == -1) r.h_hi *= 0.5;
            r.side = -1;
          } else {
            r.c_hi = cm;
            r.h_hi = h;
            CU(cudaMemcpyAsync(xhi(b), s.x, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
            TRY(save_z(zhi(b), s.z));
            if (r.side == 1) r.h_lo *= 0.5;
            r.side = 1;
          }
          TRY(illinois());
        }
      }
    }
    // grid requests waiting for their group's points
    for (int b = 0; b < L; ++b)
      if (lane_req[(size_t)b] >= 0 && !run[(size_t)b].finished && run[(size_t)b].cal == 5) TRY(group_decide(b));
    // finished requests: results out, next requests in (their lanes idle once the queue is empty)
    for (int b : freed) {
      TRY(emit(b));
      if (next_req < B) {
        TRY(assign(b));
      } else {
        lane_req[(size_t)b] = -1;
      }
    }
    TRY(kkt0_flush(c, bb));
    if (guard_iters > 1000000) return fail(MVSK_ECUDA, "batched solve did not terminate");
  }
  TRY(sync(c));
  if (infos != nullptr) {  // the per-request slots, and the free counts from W
    std::vector<double> hw((size_t)B * c->n);
    CU(cudaMemcpy(hw.data(), W_out, sizeof(double) * hw.size(), cudaMemcpyDefault));
    for (int q = 0; q < B; ++q) {
      mvsk_info& inf = infos[q];
      const double* qe = bb.q_ev + 4 * (size_t)q;
      const int* cnt = bb.q_si + (size_t)q * kSI;
      inf.krylov_iters = cnt[SI_KRY];
      inf.third_calls = cnt[SI_THIRD];
      inf.f = qe[0];
      inf.kkt_residual = qe[1];
      inf.achieved_mean = qe[2];
      inf.kkt0 = qe[3];
      inf.kkt_rel = qe[1] / fmax(qe[3], 1e-300);
      int fc = 0;
      for (int i = 0; i < c->n; ++i) fc += (hw[(size_t)q * c->n + i] - o.tau > o.eps_act);
      inf.free_count = fc;
      inf.batch_iters = (int32_t)guard_iters;
    }
  }
  return first;
}

// ------------------------------------------------ parity exports of the batch
// The direction products of one lockstep iteration on caller-given inputs
// (mvsk_batch_hvp, mvsk_batch_third): the same kernels, launch shapes and
// buffers as batch_iteration, with the operands loaded instead of produced by
// the PCG recurrences, so that tests hold them against the plain products.

// Column j < nc of instance b (b = blockIdx.y / nc) from src[(b*nc + j)*n + i]
// in FP32, zero padding to ld: PCG column j (which = 0), X column 1 + j
// (which = 1) or B column 1 + j (which = 2), the columns the products read.
__global__ void k_load_cols_f32(Inst base, int nc, int which, const double* src) {
  const int ld = base.ld, n = base.n;
  const int q = blockIdx.y, b = q / nc, j = q % nc;
  const Inst s = inst_at(base, b);
  float* col = which == 0 ? kcol<float>(s.P, j, ld) : (which == 1 ? kcol<float>(s.X, 1 + j, ld)
                                                                  : kcol<float>(s.Bv, 1 + j, ld));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ld; i += gridDim.x * blockDim.x)
    col[i] = i < n ? (float)src[((size_t)b * nc + j) * n + i] : 0.f;
}

// Instance b = blockIdx.x: c1..c4 from C[4b..4b+3] and 1/T.
__global__ void k_set_coef(Inst base, const double* C, double invT) {
  const Inst s = inst_at(base, blockIdx.x);
  if (threadIdx.x < 4) s.sd[SD_C1 + threadIdx.x] = C[4 * blockIdx.x + threadIdx.x];
  if (threadIdx.x == 0) s.sd[SD_INVT] = invT;
}

// v_b[i] = val for i < n, 0 for n <= i < ld, instance b = blockIdx.y (stride vs).
__global__ void k_fill_inst(double* v, long long vs, int n, int ld, double val) {
  double* p = v + (size_t)blockIdx.y * vs;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ld; i += gridDim.x * blockDim.x) p[i] = i < n ? val : 0.0;
}

// out[q*ld + i] = scale * sum_z part[z][q][row(i)], row(i) = upos[i] (or i
// without upos), 0 outside; z < rts[2] (or splits).  Grid-stride over N x ld.
__global__ void k_reduce_cols_u(const float* part, int splits, const int* rts, int N, int n, int ld, long long ldp,
                                double scale, const int* upos, double* out) {
  if (rts != nullptr) splits = rts[2];
  const long long tot = (long long)N * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e / ld), i = (int)(e % ld);
    const int row = i < n ? (upos != nullptr ? upos[i] : i) : -1;
    double acc = 0.0;
    if (row >= 0)
      for (int z = 0; z < splits; ++z) acc += (double)part[((size_t)z * N + q) * ldp + row];
    out[e] = scale * acc;
  }
}

// Device scratch of an export call, released when the call returns.
struct TmpDev {
  void* p = nullptr;
  ~TmpDev() {
    if (p != nullptr) cudaFree(p);
  }
  mvsk_status get(size_t bytes) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return fail(MVSK_ENOMEM, "scratch allocation of %zu bytes failed", bytes);
    }
    return MVSK_OK;
  }
};

// Instances 0..B-1 of the batch buffers at points X (B x n) with coefficients
// C (B x 4, host or device): x_b, c_b, every instance running, and the cached
// z_b = A x_b of the iteration (the FP64 streaming pass).  dev: 4B + Bn doubles.
mvsk_status batch_export_setup(mvsk_ctx* c, int B, const double* C, const double* X, double* dev) {
  BatchBuf& bb = c->batch;
  TRY(ensure_tc_pcg(c));
  TRY(batch_alloc(c, bb, B));
  const Inst& base = bb.base;
  const size_t n = (size_t)c->n;
  double* Cd = dev;
  double* Xd = dev + 4 * (size_t)B;
  CU(cudaMemcpyAsync(Cd, C, sizeof(double) * 4 * B, cudaMemcpyDefault, c->stream));
  CU(cudaMemcpyAsync(Xd, X, sizeof(double) * n * B, cudaMemcpyDefault, c->stream));
  CU(cudaMemsetAsync(base.si, 0, sizeof(int) * kSI * (size_t)B, c->stream));
  CU(cudaMemsetAsync(base.x, 0, sizeof(double) * (size_t)base.vs * B, c->stream));
  CU(cudaMemcpy2DAsync(base.x, sizeof(double) * base.vs, Xd, sizeof(double) * n, sizeof(double) * n, (size_t)B,
                       cudaMemcpyDeviceToDevice, c->stream));
  k_set_coef<<<B, 32, 0, c->stream>>>(base, Cd, 1.0 / (double)c->T);
  c->launches += 1;
  CU(cudaGetLastError());
  for (int b = 0; b < B; ++b) {
    const Inst s = inst_at(base, b);
    TRY(pass_fwd_z(c, s.x, s.z));
  }
  return MVSK_OK;
}

mvsk_status batch_hvp_export(mvsk_ctx* c, int B, const double* C, const double* X, const double* NU,
                             const double* MASK, int nc, const double* V, double* HV, double* GNU, double* DIAG,
                             int32_t* path) {
  if (c->dir_prec != P16) return fail(MVSK_EINVAL, "the batched products need a BF16 context (MVSK_PREC_MIXED_BF16)");
  if (B < 1 || B > 4096) return fail(MVSK_EINVAL, "B must be in [1, 4096]");
  if (nc < 1 || nc > kTcCols) return fail(MVSK_EINVAL, "nc must be in [1, %d]", kTcCols);
  const size_t n = (size_t)c->n, ld = (size_t)c->ld, N = (size_t)B * nc;
  TmpDev tmp;
  TRY(tmp.get(sizeof(double) * (4 * (size_t)B + 3 * n * B + N * n + N * ld)));
  double* dev = (double*)tmp.p;
  double* NUd = dev + 4 * (size_t)B + n * B;
  double* MKd = NUd + n * B;
  double* Vd = MKd + n * B;
  double* HVd = Vd + N * n;
  TRY(batch_export_setup(c, B, C, X, dev));
  BatchBuf& bb = c->batch;
  const Inst& base = bb.base;
  // the face data of the diagonal block: nuhat_b as given, the working face
  // as given (every coordinate free without a mask)
  CU(cudaMemcpyAsync(NUd, NU, sizeof(double) * n * B, cudaMemcpyDefault, c->stream));
  CU(cudaMemcpyAsync(Vd, V, sizeof(double) * n * N, cudaMemcpyDefault, c->stream));
  CU(cudaMemsetAsync(base.nuhat, 0, sizeof(double) * (size_t)base.vs * B, c->stream));
  CU(cudaMemcpy2DAsync(base.nuhat, sizeof(double) * base.vs, NUd, sizeof(double) * n, sizeof(double) * n, (size_t)B,
                       cudaMemcpyDeviceToDevice, c->stream));
  const unsigned gl = (unsigned)((ld + 255) / 256), gl4 = (unsigned)((ld + 1023) / 1024);
  k_fill_inst<<<dim3(gl, B), 256, 0, c->stream>>>(base.maskF, base.vs, c->n, c->ld, 1.0);
  c->launches += 1;
  CU(cudaGetLastError());
  if (MASK != nullptr) {
    CU(cudaMemcpyAsync(MKd, MASK, sizeof(double) * n * B, cudaMemcpyDefault, c->stream));
    CU(cudaMemcpy2DAsync(base.maskF, sizeof(double) * base.vs, MKd, sizeof(double) * n, sizeof(double) * n,
                         (size_t)B, cudaMemcpyDeviceToDevice, c->stream));
  }
  bb.umode = c->opt.face_products != 0;
  int s2 = 0, fused = 0;
  const int* rts = nullptr;
  if (bb.umode) {  // the products restricted to the union of the given faces
    TRY(ensure_ubuf(c, bb));
    TRY(u_prepare(c, bb, B, &nc, 1, 0));
    TRY(union_gather(c, bb, B));
    TRY(hvpdiag_tc_batch_u(c, bb, B, oz_row_ctas(c)));
    k_load_cols_f32<<<dim3(gl, (unsigned)N), 256, 0, c->stream>>>(base, nc, 0, Vd);
    k_cols_bf16_u<<<dim3(gl, (unsigned)N), 256, 0, c->stream>>>(base, nc, 0, 0, bb.u_idx, bb.u_info, bb.P16);
    c->launches += 2;
    CU(cudaGetLastError());
    fused = u_fused(c, (int)N) ? 1 : 0;
    TRY(hvp_tc_batch_u(c, bb, B, nc, &rts));
  } else {
    TRY(hvpdiag_tc_batch(c, bb, B, oz_row_ctas(c)));
    k_load_cols_f32<<<dim3(gl, (unsigned)N), 256, 0, c->stream>>>(base, nc, 0, Vd);
    k_cols_bf16_b<<<dim3(gl4, (unsigned)N), 256, 0, c->stream>>>(base, nc, 0, 0, bb.P16);
    c->launches += 2;
    CU(cudaGetLastError());
    TRY(hvp_tc_batch(c, bb, B, nc, &s2, &fused));
  }
  k_reduce_cols_u<<<4 * c->nsm, 256, 0, c->stream>>>(bb.part, s2, rts, (int)N, c->n, c->ld, c->ld,
                                                     1.0 / (double)c->T, bb.umode ? bb.u_pos : nullptr, HVd);
  c->launches += 1;
  CU(cudaGetLastError());
  if (rts != nullptr) CU(cudaMemcpyAsync(&s2, rts + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpy2DAsync(HV, sizeof(double) * n, HVd, sizeof(double) * ld, sizeof(double) * n, N, cudaMemcpyDefault,
                       c->stream));
  CU(cudaMemcpy2DAsync(GNU, sizeof(double) * n, base.Gnu, sizeof(double) * 2 * base.vs, sizeof(double) * n,
                       (size_t)B, cudaMemcpyDefault, c->stream));
  CU(cudaMemcpy2DAsync(DIAG, sizeof(double) * n, base.diagG, sizeof(double) * 2 * base.vs, sizeof(double) * n,
                       (size_t)B, cudaMemcpyDefault, c->stream));
  TRY(sync(c));
  if (path != nullptr) {
    path[0] = fused;
    path[1] = s2;
  }
  return MVSK_OK;
}

mvsk_status batch_third_export(mvsk_ctx* c, int B, const double* C, const double* X, const double* MASK, int K,
                               const double* U, const double* P, double* AT) {
  if (c->dir_prec != P16) return fail(MVSK_EINVAL, "the batched products need a BF16 context (MVSK_PREC_MIXED_BF16)");
  if (B < 1 || B > 4096) return fail(MVSK_EINVAL, "B must be in [1, 4096]");
  if (K < 1 || 2 * K > kTcCols) return fail(MVSK_EINVAL, "K must be in [1, %d]", kTcCols / 2);
  const size_t n = (size_t)c->n, ld = (size_t)c->ld, NK = (size_t)B * K;
  TmpDev tmp;
  TRY(tmp.get(sizeof(double) * (4 * (size_t)B + 2 * n * B + 2 * NK * n)));
  double* dev = (double*)tmp.p;
  double* MKd = dev + 4 * (size_t)B + n * B;
  double* Ud = MKd + n * B;
  double* Pd = Ud + NK * n;
  TRY(batch_export_setup(c, B, C, X, dev));
  BatchBuf& bb = c->batch;
  const Inst& base = bb.base;
  CU(cudaMemcpyAsync(Ud, U, sizeof(double) * n * NK, cudaMemcpyDefault, c->stream));
  CU(cudaMemcpyAsync(Pd, P, sizeof(double) * n * NK, cudaMemcpyDefault, c->stream));
  const unsigned gl = (unsigned)((ld + 255) / 256);
  k_fill_inst<<<dim3(gl, B), 256, 0, c->stream>>>(base.maskF, base.vs, c->n, c->ld, 1.0);
  k_load_cols_f32<<<dim3(gl, (unsigned)NK), 256, 0, c->stream>>>(base, K, 1, Ud);
  k_load_cols_f32<<<dim3(gl, (unsigned)NK), 256, 0, c->stream>>>(base, K, 2, Pd);
  c->launches += 3;
  CU(cudaGetLastError());
  if (MASK != nullptr) {
    CU(cudaMemcpyAsync(MKd, MASK, sizeof(double) * n * B, cudaMemcpyDefault, c->stream));
    CU(cudaMemcpy2DAsync(base.maskF, sizeof(double) * base.vs, MKd, sizeof(double) * n, sizeof(double) * n,
                         (size_t)B, cudaMemcpyDeviceToDevice, c->stream));
  }
  bb.umode = c->opt.face_products != 0;
  if (bb.umode) {
    TRY(ensure_ubuf(c, bb));
    const int one = 1;
    TRY(u_prepare(c, bb, B, &one, 1, K));
    TRY(union_gather(c, bb, B));
    int mode = 0;  // the small-face block's kernels when every face allows them (option face_small)
    if (c->opt.face_small) {
      k_face_list<<<dim3(1, B), 1024, 0, c->stream>>>(base, bb.f_list);
      k_small_mode<<<1, 256, 0, c->stream>>>(base, B, 1, c->opt.face_small == 2, bb.u_info, 0, 0);
      c->launches += 2;
      CU(cudaGetLastError());
      CU(cudaMemcpyAsync(&mode, bb.u_info + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      TRY(sync(c));
    }
    if (mode == 2) {
      TRY(small_face_third<kMFt>(c, bb, B, K));
    } else if (mode == 1) {
      TRY(small_face_third<kMF>(c, bb, B, K));
    } else {
      TRY(third_tc_batch_u(c, bb, B, K));
    }
  } else {
    TRY(third_tc_batch(c, bb, B, K));
  }
  CU(cudaMemcpy2DAsync(AT, sizeof(double) * n, base.at, sizeof(double) * base.vs, sizeof(double) * n, (size_t)B,
                       cudaMemcpyDefault, c->stream));
  return sync(c);
}
