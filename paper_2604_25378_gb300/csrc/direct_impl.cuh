// Direct configuration of the affine-normal block (Sec. 3.2, Table
// yand-core-parameters "direct reduced solve"), included into mvsk_api.cu.
//
// On the working face F with C = [1_F/sqrt(m), nu] (orthonormal) and
// P = I_F - C C^T:
//   G = T^-1 A^T Diag(psi''(z)) A                          (Prop. 2)
//   B = P (G_FF + lambda I) P + s C C^T  on F, identity off F
// B restricted to V = range(P) is H_{T,lambda} in any orthonormal basis of V,
// so B is positive definite iff H is, and S = P B^-1 P = M H^-1 M^T.  Then
//   u_h = S h, h = P G nu;   r_t = a_t^T S a_t (exact trace, reading S5);
//   a = P T^-1 A^T (psi'''(z) o r);   d = u_h - (||gbar||/m) S a - nu.
// B^-1 comes from a block Gauss-Jordan sweep whose pivot blocks are Cholesky-
// factored (a failing pivot means B is not positive definite and the next
// regularisation of the fallback list is tried).  s = |tr P G P|/(m-2) keeps
// the C C^T block on the scale of H.
#pragma once

__global__ void k_psi2_vec(const double* z, long long T, double c2, double c3, double c4, double* out) {
  const Psi psi{c2, c3, c4};
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (long long)gridDim.x * blockDim.x)
    out[t] = psi.d2(z[t]);
}

// y_i = sum_j M[i*ld + j] x_j for i < n (one warp per row); rows with mask 0 give 0.
__global__ void k_matvec(const double* Mx, int ld, int n, const double* x, const double* mask, double* y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += Mx[(size_t)warp * ld + j] * x[j];
  s = warp_sum(s);
  if (lane == 0) y[warp] = (mask == nullptr || mask[warp] != 0.0) ? s : 0.0;
}

// r_t = sum_j Y[t][j] A[t][j] (one warp per row).
__global__ void k_rowdot(const double* Y, const double* A, long long T, int ld, int n, double* r) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= T) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += Y[(size_t)warp * ld + j] * A[(size_t)warp * ld + j];
  s = warp_sum(s);
  if (lane == 0) r[warp] = s;
}

// lambda = reg |tr P G P| / (m-2) and the C C^T scale s (slots SD_LAM, SD_SUMZ2).
__global__ void __launch_bounds__(kVT) k_direct_lambda(Inst s, const double* G, int ld, const double* GC, double reg) {
  __shared__ double scr[80];
  const int n = s.n;
  const double m = (double)s.si[SI_M];
  const double r1 = 1.0 / sqrt(m);
  double tr = 0.0, c11 = 0.0, c22 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (s.maskF[i] != 0.0) tr += G[(size_t)i * ld + i];
    c11 += s.maskF[i] * r1 * GC[i];
    c22 += s.nuhat[i] * GC[ld + i];
  }
  const double2 a = block_sum2(tr, c11, scr);
  const double c22s = block_sum2(c22, 0.0, scr).x;
  if (threadIdx.x == 0) {
    const double t = fabs(a.x - a.y - c22s) / (m - 2.0);
    s.sd[SD_LAM] = reg * t;
    s.sd[SD_SUMZ2] = t > 0.0 ? t : 1.0;
  }
}

// B_ij of the face matrix (see the file comment); ld x ld with zero padding.
__global__ void k_build_B(Inst s, const double* G, int ld, const double* GC, double* Bm) {
  const int n = s.n;
  const double m = (double)s.si[SI_M];
  const double lam = s.sd[SD_LAM], sc = s.sd[SD_SUMZ2];
  const double r1 = 1.0 / sqrt(m);
  // C^T G C (2 x 2) is recomputed per block from GC: cheap (n terms) and avoids a launch
  __shared__ double cgc[3];
  __shared__ double scr[80];
  double a11 = 0.0, a12 = 0.0, a22 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double u1 = s.maskF[i] * r1, u2 = s.nuhat[i];
    a11 += u1 * GC[i];
    a12 += u1 * GC[ld + i];
    a22 += u2 * GC[ld + i];
  }
  const double2 p = block_sum2(a11, a12, scr);
  const double q = block_sum2(a22, 0.0, scr).x;
  if (threadIdx.x == 0) {
    cgc[0] = p.x + lam;
    cgc[1] = p.y;
    cgc[2] = q + lam;
  }
  __syncthreads();
  const long long tot = (long long)ld * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), j = (int)(e % ld);
    double v = 0.0;
    if (i < n && j < n) {
      const bool fi = s.maskF[i] != 0.0, fj = s.maskF[j] != 0.0;
      if (fi && fj) {
        const double ui1 = r1, ui2 = s.nuhat[i], uj1 = r1, uj2 = s.nuhat[j];
        const double ki1 = GC[i] + lam * ui1, ki2 = GC[ld + i] + lam * ui2;
        const double kj1 = GC[j] + lam * uj1, kj2 = GC[ld + j] + lam * uj2;
        v = G[(size_t)i * ld + j] + (i == j ? lam : 0.0);
        v -= ki1 * uj1 + ki2 * uj2;
        v -= ui1 * kj1 + ui2 * kj2;
        v += ui1 * (cgc[0] * uj1 + cgc[1] * uj2) + ui2 * (cgc[1] * uj1 + cgc[2] * uj2);
        v += sc * (ui1 * uj1 + ui2 * uj2);
      } else if (i == j && !fi) {
        v = 1.0;
      }
    }
    Bm[e] = v;
  }
}

// S = P B^-1 P = B^-1 - (1/s) C C^T on F, zero elsewhere (in place).
__global__ void k_make_S(Inst s, int ld, double* Bm) {
  const int n = s.n;
  const double m = (double)s.si[SI_M];
  const double r1 = 1.0 / sqrt(m), isc = 1.0 / s.sd[SD_SUMZ2];
  const long long tot = (long long)ld * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), j = (int)(e % ld);
    double v = 0.0;
    if (i < n && j < n && s.maskF[i] != 0.0 && s.maskF[j] != 0.0)
      v = Bm[e] - isc * (r1 * r1 + s.nuhat[i] * s.nuhat[j]);
    Bm[e] = v;
  }
}

// v <- P_V v in place (one CTA).
__global__ void __launch_bounds__(kVT) k_project_V(Inst s, double* v) {
  __shared__ double scr[80];
  project_V(v, v, s.maskF, s.nuhat, s.n, (double)s.si[SI_M], scr);
}

mvsk_status gemm64(mvsk_ctx* c, bool at, bool bt, int M, int N, int K, double alpha, const double* A, long long lda,
                   const double* B, long long ldb, const double* sk, double beta, double* C, long long ldc) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  if (grid.y > 65535) return fail(MVSK_EINVAL, "dense product too tall (%d rows)", M);
  c->launches += 1;
  if (!at && !bt) k_dgemm<false, false><<<grid, 256, 0, c->stream>>>(M, N, K, alpha, A, lda, B, ldb, sk, beta, C, ldc);
  else if (!at && bt) k_dgemm<false, true><<<grid, 256, 0, c->stream>>>(M, N, K, alpha, A, lda, B, ldb, sk, beta, C, ldc);
  else if (at && !bt) k_dgemm<true, false><<<grid, 256, 0, c->stream>>>(M, N, K, alpha, A, lda, B, ldb, sk, beta, C, ldc);
  else k_dgemm<true, true><<<grid, 256, 0, c->stream>>>(M, N, K, alpha, A, lda, B, ldb, sk, beta, C, ldc);
  CU(cudaGetLastError());
  return MVSK_OK;
}

mvsk_status ensure_direct_buffers(mvsk_ctx* c) {
  if (c->Gm != nullptr) return MVSK_OK;
  const size_t ld = (size_t)c->ld;
  void* p;
  TRY(dalloc(c, &p, sizeof(double) * ld * ld));
  c->Gm = (double*)p;
  TRY(dalloc(c, &p, sizeof(double) * ld * ld));
  c->Bm = (double*)p;
  TRY(dalloc(c, &p, sizeof(double) * ld * 64));
  c->Ub = (double*)p;
  TRY(dalloc(c, &p, sizeof(double) * ld * 64));
  c->Rb = (double*)p;
  TRY(dalloc(c, &p, sizeof(double) * 64 * 64));
  c->Pb = (double*)p;
  TRY(dalloc(c, &p, sizeof(double) * 2 * ld));
  c->GC = (double*)p;
  TRY(dalloc(c, &p, sizeof(double) * (size_t)c->T * ld));
  c->Yb = (double*)p;
  TRY(dalloc(c, &p, sizeof(double) * (size_t)c->T));
  c->dvec = (double*)p;
  TRY(dalloc(c, &p, 64));
  c->dflag = (int*)p;
  return MVSK_OK;
}

// Weighted Gram G = T^-1 A^T Diag(psi''(z)) A into c->Gm (ld x ld, n x n used):
// FP64 SIMT from the FP64 master copy, or BF16 x BF16 -> FP32 on the tensor
// cores (tcgen05) from A^T and (Diag(psi'') A)^T in BF16 when prec = P16.
mvsk_status gram_into(mvsk_ctx* c, const double* z, int prec) {
  TRY(ensure_direct_buffers(c));
  c->launches += 1;
  k_psi2_vec<<<4 * c->nsm, 256, 0, c->stream>>>(z, c->T, c->c[1], c->c[2], c->c[3], c->dvec);
  CU(cudaGetLastError());
  if (prec == P16) {
    TRY(ensure_tc_operands(c));
    TRY(transpose_bf16(c, c->dvec, c->W16T));
    return gemm_tc_f64(c, c->A16T, c->n, c->W16T, c->n, c->T, c->Tp, 1.0 / (double)c->T, c->Gm, c->ld);
  }
  return gemm64(c, true, true, c->n, c->n, (int)c->T, 1.0 / (double)c->T, c->A64, c->ld, c->A64, c->ld, c->dvec, 0.0,
                c->Gm, c->ld);
}

// B^-1 in place by the block Gauss-Jordan sweep; returns whether B was positive definite.
mvsk_status sweep_inverse(mvsk_ctx* c, bool* pd) {
  const int n = c->n, ld = c->ld;
  double* Bm = c->Bm;
  CU(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->stream));
  for (int k0 = 0; k0 < n; k0 += 64) {
    const int b = n - k0 < 64 ? n - k0 : 64;
    k_pivot_inverse<<<1, 256, 0, c->stream>>>(Bm, ld, k0, b, c->Pb, c->dflag);
    k_copy_block<<<c->nsm, 256, 0, c->stream>>>(Bm + k0, ld, c->Ub, 64, n, b, 1.0, k0, k0 + b);
    c->launches += 2;
    CU(cudaGetLastError());
    TRY(gemm64(c, false, true, b, n, b, 1.0, c->Pb, b, Bm + (size_t)k0 * ld, ld, nullptr, 0.0, c->Rb, ld));
    k_copy_block<<<c->nsm, 256, 0, c->stream>>>(c->Rb, ld, Bm + (size_t)k0 * ld, ld, b, n, 1.0, 0, 0);
    c->launches += 1;
    TRY(gemm64(c, false, true, n, n, b, -1.0, c->Ub, 64, c->Rb, ld, nullptr, 1.0, Bm, ld));
    TRY(gemm64(c, false, true, n, b, b, -1.0, c->Ub, 64, c->Pb, b, nullptr, 0.0, Bm + k0, ld));
    k_copy_block<<<1, 256, 0, c->stream>>>(c->Pb, b, Bm + (size_t)k0 * ld + k0, ld, b, b, 1.0, 0, 0);
    c->launches += 1;
    CU(cudaGetLastError());
  }
  int flag = 0;
  CU(cudaMemcpyAsync(&flag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  TRY(sync(c));
  *pd = flag == 0;
  return MVSK_OK;
}

mvsk_status direction_direct(mvsk_ctx* c) {
  Inst& s = c->in;
  int h2[2];
  TRY(read_ints(c, h2, SI_DONE, 1));
  TRY(read_ints(c, h2 + 1, SI_SKIPDIR, 1));
  if (h2[0] != 0 || h2[1] != 0) return MVSK_OK;
  const int n = c->n, ld = c->ld;
  TRY(gram_into(c, s.z, c->dir_prec == P16 ? P16 : P64));
  // G C (two columns: 1_F/sqrt(m) and nu); the mask vector is 1_F
  const int mvb = (n * 32 + 255) / 256;
  k_matvec<<<mvb, 256, 0, c->stream>>>(c->Gm, ld, n, s.maskF, s.maskF, c->GC);
  k_matvec<<<mvb, 256, 0, c->stream>>>(c->Gm, ld, n, s.nuhat, s.maskF, c->GC + ld);
  c->launches += 2;
  CU(cudaGetLastError());
  // GC[0..n) holds G 1_F; scale it to G (1_F / sqrt(m)) in place
  int mh = 0;
  TRY(read_ints(c, &mh, SI_M, 1));
  k_copy_block<<<c->nsm, 256, 0, c->stream>>>(c->GC, ld, c->GC, ld, 1, n, 1.0 / sqrt((double)mh), 0, 0);
  c->launches += 1;
  CU(cudaGetLastError());
  const double reg0 = isnan(c->opt.reg) ? 0.0 : c->opt.reg;
  std::vector<double> regs = {reg0};
  for (double r : {1e-4, 1e-2})
    if (r > reg0) regs.push_back(r);
  bool pd = false;
  for (double rg : regs) {
    k_direct_lambda<<<1, kVT, 0, c->stream>>>(s, c->Gm, ld, c->GC, rg);
    k_build_B<<<4 * c->nsm, 256, 0, c->stream>>>(s, c->Gm, ld, c->GC, c->Bm);
    c->launches += 2;
    CU(cudaGetLastError());
    TRY(sweep_inverse(c, &pd));
    if (pd) break;
  }
  if (!pd) {  // every regularisation failed: d = -nu
    CU(cudaMemcpyAsync(s.d, s.nuhat, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
    k_copy_block<<<1, 256, 0, c->stream>>>(s.d, ld, s.d, ld, 1, n, -1.0, 0, 0);
    c->launches += 1;
    CU(cudaGetLastError());
    return MVSK_OK;
  }
  k_make_S<<<4 * c->nsm, 256, 0, c->stream>>>(s, ld, c->Bm);
  // h = P G nu ; u_h = S h  (stored as PCG column 0 so k_assemble can be reused)
  double* h = s.Bv;
  double* uh = s.X;
  k_matvec<<<mvb, 256, 0, c->stream>>>(c->Gm, ld, n, s.nuhat, s.maskF, h);
  k_project_V<<<1, kVT, 0, c->stream>>>(s, h);
  k_matvec<<<mvb, 256, 0, c->stream>>>(c->Bm, ld, n, h, nullptr, uh);
  c->launches += 4;
  CU(cudaGetLastError());
  // exact trace: r_t = a_t^T S a_t via Y = A S
  TRY(gemm64(c, false, false, (int)c->T, n, n, 1.0, c->A64, ld, c->Bm, ld, nullptr, 0.0, c->Yb, ld));
  const long long rb = (c->T * 32 + 255) / 256;
  k_rowdot<<<(unsigned)rb, 256, 0, c->stream>>>(c->Yb, c->A64, c->T, ld, n, s.rhat);
  c->launches += 1;
  CU(cudaGetLastError());
  // a = P T^-1 A^T (psi''' o r)
  {
    PassArgs a = pass_args(c);
    a.z = s.z;
    a.roww = s.rhat;
    TRY(run_pass(c, P64, M_BACK, 0, a));
    TRY(reduce_cols(c, P64, 1, s.at, ld, nullptr, 0.0, nullptr, nullptr));
  }
  k_project_V<<<1, kVT, 0, c->stream>>>(s, s.at);
  const int ca = c->ncolmax - 1;
  k_matvec<<<mvb, 256, 0, c->stream>>>(c->Bm, ld, n, s.at, nullptr, s.X + (size_t)ca * ld);
  k_assemble<double><<<1, kVT, 0, c->stream>>>(s, ca);
  c->launches += 3;
  CU(cudaGetLastError());
  return MVSK_OK;
}
