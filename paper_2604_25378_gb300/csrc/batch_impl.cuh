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
// dst[(b*nc + j)*ld + i] = bf16(col_j of instance b): PCG column c0 + j, or the
// interleaved (X_{1+k}, B_{1+k}) pairs when interleave != 0.
__global__ void k_cols_bf16_b(Inst base, int B, int c0, int nc, int interleave, __nv_bfloat16* dst) {
  const int ld = base.ld;
  const long long tot = (long long)B * nc * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % ld);
    const long long q = e / ld;
    const int b = (int)(q / nc), j = (int)(q % nc);
    const Inst s = inst_at(base, b);
    double v;
    if (interleave) v = (j & 1) ? s.Bv[(size_t)(1 + (j >> 1)) * ld + i] : s.X[(size_t)(1 + (j >> 1)) * ld + i];
    else v = s.P[(size_t)(c0 + j) * ld + i];
    dst[e] = __float2bfloat16((float)v);
  }
}

// S^T[q][t] = bf16(psi''_b(z_b[t]) * sum_z part[z][q][t]), b = q / nc.
__global__ void k_reduce_hvp1_b(const float* part, int splits, int N, int nc, long long T, long long ldp, Inst base,
                                __nv_bfloat16* S, long long Tp) {
  const long long tot = (long long)N * T;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e / T);
    const long long t = e % T;
    const Inst s = inst_at(base, q / nc);
    float acc = 0.f;
    for (int z = 0; z < splits; ++z) acc += part[((size_t)z * N + q) * ldp + t];
    const Psi psi{s.sd[SD_C2], s.sd[SD_C3], s.sd[SD_C4]};
    S[(size_t)q * Tp + t] = __float2bfloat16((float)(psi.d2(s.z[t]) * (double)acc));
  }
}

// Q_b[c0 + j][i] = T^-1 sum_z part[z][b*nc + j][i] (i < n; zero padding to ld).
// mode 1 writes the single column to at_b instead (back-projection of a).
__global__ void k_reduce_hvp2_b(const float* part, int splits, int N, int nc, int n, int ld, long long ldp,
                                double scale, Inst base, int c0, int mode) {
  const long long tot = (long long)N * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e / ld), i = (int)(e % ld);
    const Inst s = inst_at(base, q / nc);
    double acc = 0.0;
    if (i < n)
      for (int z = 0; z < splits; ++z) acc += (double)part[((size_t)z * N + q) * ldp + i];
    if (mode == 1) s.at[i] = scale * acc;
    else s.Q[(size_t)(c0 + q % nc) * ld + i] = scale * acc;
  }
}

// rhat_b[t] = K^-1 sum_k (A X_k)_t (A p_k)_t; S^T[b][t] = bf16(psi3_b(z_b[t]) rhat_b[t]).
__global__ void k_reduce_rhat_b(const float* part, int splits, int N, int K, long long T, long long ldp, Inst base,
                                __nv_bfloat16* S, long long Tp) {
  const int B = N / (2 * K);
  const long long tot = (long long)B * T;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / T);
    const long long t = e % T;
    const Inst s = inst_at(base, b);
    double r = 0.0;
    for (int k = 0; k < K; ++k) {
      float u = 0.f, v = 0.f;
      const int q = b * 2 * K + 2 * k;
      for (int z = 0; z < splits; ++z) {
        u += part[((size_t)z * N + q) * ldp + t];
        v += part[((size_t)z * N + q + 1) * ldp + t];
      }
      r += (double)u * (double)v;
    }
    r /= K;
    s.rhat[t] = r;
    const Psi psi{0.0, s.sd[SD_C3], s.sd[SD_C4]};
    S[(size_t)b * Tp + t] = __float2bfloat16((float)(psi.d3(s.z[t]) * r));
  }
}

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
  bb.cap = B;
  return MVSK_OK;
}

// Split-K tensor-core product with FP32 partials for N columns (N tile 16, 64 or 256).
mvsk_status tc_partials_n(mvsk_ctx* c, const void* Aop, int M, const void* Bop, int N, long long K, long long ldk,
                          float* part, size_t part_floats, long long ldp, int* splits_out) {
  CUtensorMap ta, tb;
  const int bn = N <= 16 ? 16 : (N <= 64 ? 64 : 256);
  TRY(make_tmap_bf16(&ta, Aop, (unsigned long long)ldk, (unsigned long long)M, (unsigned long long)ldk * 2, kTcBK,
                     kTcBM));
  TRY(make_tmap_bf16(&tb, Bop, (unsigned long long)ldk, (unsigned long long)N, (unsigned long long)ldk * 2, kTcBK,
                     (unsigned)bn));
  const int mt = (M + kTcBM - 1) / kTcBM, nt = (N + bn - 1) / bn;
  const int nk = (int)((K + kTcBK - 1) / kTcBK);
  int want = (2 * c->nsm + mt * nt - 1) / (mt * nt);
  const int maxs = (int)(part_floats / ((size_t)N * ldp));
  if (want > maxs) want = maxs;
  if (want > 8) want = 8;
  if (want > nk) want = nk;
  if (want < 1) want = 1;
  const int ktps = (nk + want - 1) / want;
  const int splits = (nk + ktps - 1) / ktps;
  EpiPartT epi{part, ldp, M, N};
  dim3 grid((unsigned)nt, (unsigned)mt, (unsigned)splits);
  TRY(prof_begin(c, 400 + bn, 2.0 * (double)M * (double)N * (double)K));
  if (bn == 16)
    k_gemm_tc<16, 8, EpiPartT><<<grid, 128, tc_smem_bytes<16, 8>(), c->stream>>>(ta, tb, M, N, (int)K, ktps, epi,
                                                                                c->err, nullptr, nullptr);
  else if (bn == 64)
    k_gemm_tc<64, 6, EpiPartT><<<grid, 128, tc_smem_bytes<64, 6>(), c->stream>>>(ta, tb, M, N, (int)K, ktps, epi,
                                                                                c->err, nullptr, nullptr);
  else
    k_gemm_tc<256, 4, EpiPartT><<<grid, 128, tc_smem_bytes<256, 4>(), c->stream>>>(ta, tb, M, N, (int)K, ktps, epi,
                                                                                  c->err, nullptr, nullptr);
  c->launches += 1;
  CU(cudaGetLastError());
  TRY(prof_end(c));
  *splits_out = splits;
  return MVSK_OK;
}

// Q_b[c0..c0+nc) = T^-1 A^T (psi''_b(z_b) o A P_b[c0..c0+nc)) for every instance.
mvsk_status hvp_tc_batch(mvsk_ctx* c, BatchBuf& bb, int B, int c0, int nc) {
  const int N = B * nc, gb = 4 * c->nsm;
  k_cols_bf16_b<<<gb, 256, 0, c->stream>>>(bb.base, B, c0, nc, 0, bb.P16);
  int s1 = 0, s2 = 0;
  TRY(tc_partials_n(c, c->Alo, (int)c->T, bb.P16, N, c->ld, c->ld, bb.part, bb.part_floats, c->T, &s1));
  k_reduce_hvp1_b<<<gb, 256, 0, c->stream>>>(bb.part, s1, N, nc, c->T, c->T, bb.base, bb.S16T, c->Tp);
  TRY(tc_partials_n(c, c->A16T, c->n, bb.S16T, N, c->Tp, c->Tp, bb.part, bb.part_floats, c->ld, &s2));
  k_reduce_hvp2_b<<<gb, 256, 0, c->stream>>>(bb.part, s2, N, nc, c->n, c->ld, c->ld, 1.0 / (double)c->T, bb.base, c0,
                                             0);
  c->launches += 3;
  CU(cudaGetLastError());
  return MVSK_OK;
}

// rhat_b and at_b = T^-1 A^T (psi3_b(z_b) o rhat_b) for every instance.
mvsk_status third_tc_batch(mvsk_ctx* c, BatchBuf& bb, int B, int K) {
  const int N = B * 2 * K, gb = 4 * c->nsm;
  k_cols_bf16_b<<<gb, 256, 0, c->stream>>>(bb.base, B, 0, 2 * K, 1, bb.P16);
  int s1 = 0, s2 = 0;
  TRY(tc_partials_n(c, c->Alo, (int)c->T, bb.P16, N, c->ld, c->ld, bb.part, bb.part_floats, c->T, &s1));
  k_reduce_rhat_b<<<gb, 256, 0, c->stream>>>(bb.part, s1, N, K, c->T, c->T, bb.base, bb.S16T, c->Tp);
  TRY(tc_partials_n(c, c->A16T, c->n, bb.S16T, B, c->Tp, c->Tp, bb.part, bb.part_floats, c->ld, &s2));
  k_reduce_hvp2_b<<<gb, 256, 0, c->stream>>>(bb.part, s2, B, 1, c->n, c->ld, c->ld, 1.0 / (double)c->T, bb.base, 0, 1);
  c->launches += 3;
  CU(cudaGetLastError());
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
mvsk_status batch_iteration(mvsk_ctx* c, BatchBuf& bb, int B, const std::vector<std::array<double, 4>>& cc) {
  const Inst& base = bb.base;
  const int K = c->opt.probes, ncol1 = K + 1, ca = K + 1, kmax = c->opt.krylov_maxit;
  const int P = c->dir_prec;
  for (int b = 0; b < B; ++b) {
    const Inst s = inst_at(base, b);
    PassArgs a = pass_args_inst(cc[b].data());
    a.in[0] = s.x;
    a.rowout = s.z;
    a.skip = s.si + SI_DONE;
    TRY(run_pass(c, P64, M_VALGRAD, 1, a, nullptr, s.spart));
    TRY(reduce_cols(c, P64, 1, s.g, c->ld, c->mu, 0.0, s.si + SI_DONE, nullptr, s.sd + SD_C1));
  }
  k_face<<<dim3(1, B), kVT, 0, c->stream>>>(base, nullptr, c->grid);
  c->launches += 1;
  CU(cudaGetLastError());
  for (int b = 0; b < B; ++b) {
    const Inst s = inst_at(base, b);
    PassArgs a = pass_args_inst(cc[b].data());
    a.in[0] = s.nuhat;
    a.in[1] = s.maskF;
    a.z = s.z;
    a.skip = s.si + SI_SKIPDIR;
    TRY(run_pass(c, P, M_HVPDIAG, 2, a, nullptr, s.spart));
    TRY(reduce_cols(c, P, 2, s.Gnu, c->ld, nullptr, 0.0, s.si + SI_SKIPDIR, nullptr));
  }
  if (K > 0) k_probe_fill<<<dim3((c->ld + 255) / 256, K, B), 256, 0, c->stream>>>(base, K);
  k_pcg_setup<<<dim3(1, B), kVT, 0, c->stream>>>(base, nullptr, c->grid, (ncol1 + 1) / 2);
  c->launches += 2;
  CU(cudaGetLastError());
  for (int it = 0; it < kmax; ++it) {
    TRY(hvp_tc_batch(c, bb, B, 0, ncol1));
    k_pcg_step<<<dim3(ncol1, B), kPT, 0, c->stream>>>(base, 0, kmax);
    c->launches += 1;
    CU(cudaGetLastError());
  }
  if (K > 0) {
    TRY(third_tc_batch(c, bb, B, K));
  } else {
    for (int b = 0; b < B; ++b) CU(cudaMemsetAsync(inst_at(base, b).at, 0, sizeof(double) * c->ld, c->stream));
  }
  k_pcg_setup2<<<dim3(1, B), kVT, 0, c->stream>>>(base, ca, ca / 2);
  c->launches += 1;
  CU(cudaGetLastError());
  for (int it = 0; it < kmax; ++it) {
    TRY(hvp_tc_batch(c, bb, B, ca, 1));
    k_pcg_step<<<dim3(1, B), kPT, 0, c->stream>>>(base, ca, kmax);
    c->launches += 1;
    CU(cudaGetLastError());
  }
  k_assemble<<<dim3(1, B), kVT, 0, c->stream>>>(base, ca);
  c->launches += 1;
  CU(cudaGetLastError());
  for (int b = 0; b < B; ++b) {
    const Inst s = inst_at(base, b);
    PassArgs a = pass_args_inst(cc[b].data());
    a.in[0] = s.d;
    a.z = s.z;
    a.skip = s.si + SI_DONE;
    TRY(run_pass(c, P64, M_LS, 1, a, nullptr, s.spart));
  }
  k_decide1<<<dim3(1, B), kVT, 0, c->stream>>>(base, nullptr, c->grid);
  c->launches += 1;
  CU(cudaGetLastError());
  for (int b = 0; b < B; ++b) {
    const Inst s = inst_at(base, b);
    PassArgs a = pass_args_inst(cc[b].data());
    a.in[0] = s.dstep;
    a.z = s.z;
    a.skip = s.si + SI_SKIPLS;
    TRY(run_pass(c, P64, M_LS, 1, a, nullptr, s.spart));
  }
  k_decide2<<<dim3(1, B), kVT, 0, c->stream>>>(base, nullptr, c->grid);
  k_end_iter<<<dim3(1, B), 32, 0, c->stream>>>(base);
  c->launches += 2;
  CU(cudaGetLastError());
  return MVSK_OK;
}

// Per-instance host state: stall-recovery phases and the target calibration.
struct InstRun {
  double lam[4] = {0, 0, 0, 0}, target = NAN;
  std::array<double, 4> cc{};
  int phase = 0;
  int cal = 0;  // 0 no target, 1 lower-end solve, 2 growing, 3 Illinois
  double c_lo = 0, c_hi = 0, h_lo = 0, h_hi = 0, c1_ref = 0, c1_max = 0;
  int side = 0, evals = 0, iters = 0, restarts = 0;
  int run_status = MVSK_OK;
  bool finished = false, final_from_hi = false;
  std::chrono::steady_clock::time_point t_start;
  double ev[3] = {0, 0, 0};
};

// Start an inner solve of instance b at c1 from warm start w0 (device vector or null).
mvsk_status batch_start_run(mvsk_ctx* c, BatchBuf& bb, int b, InstRun& r, double c1, const double* w0, double tol) {
  const Inst s = inst_at(bb.base, b);
  r.cc[0] = c1;
  const Options& o = c->opt;
  const double reg = isnan(o.reg) ? 1e-4 : o.reg;
  double h[12] = {o.tau, o.eps_act, o.release_ratio, reg, o.krylov_tol, r.cc[0], r.cc[1], r.cc[2], r.cc[3],
                  1.0 / (double)c->T, o.descent_eps, o.stall_factor};
  double* dopts = s.tmp + (size_t)22 * c->ld;  // 12 doubles of the instance's scratch
  CU(cudaMemcpyAsync(dopts, h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  k_init_state<<<1, 32, 0, c->stream>>>(s, tol, o.eta, o.pcg_max_iter, 1, o.stall_window, o.probes, o.probe_seed,
                                        o.krylov_maxit, o.arc_halvings, dopts);
  k_fill<<<(c->ld + 255) / 256, 256, 0, c->stream>>>(s.x, c->n, c->ld, 1.0 / c->n);
  PassArgs a = pass_args_inst(r.cc.data());
  a.in[0] = s.x;
  a.rowout = s.z;
  TRY(run_pass(c, P64, M_VALGRAD, 1, a, nullptr, s.spart));
  TRY(reduce_cols(c, P64, 1, s.g, c->ld, c->mu, -c1, nullptr, nullptr));
  k_kkt0<<<1, kVT, 0, c->stream>>>(s);
  if (w0 != nullptr) CU(cudaMemcpyAsync(s.x, w0, sizeof(double) * c->ld, cudaMemcpyDeviceToDevice, c->stream));
  k_new_phase<<<1, 32, 0, c->stream>>>(s, o.eta, o.pcg_max_iter);
  c->launches += 5;
  CU(cudaGetLastError());
  r.phase = 0;
  r.evals += 1;
  r.t_start = std::chrono::steady_clock::now();
  return MVSK_OK;
}

mvsk_status batch_solve(mvsk_ctx* c, int B, const double* lam_h, const double* tg_h, double tol, const double* W0,
                        double* W_out, mvsk_info* infos) {
  BatchBuf& bb = c->batch;
  TRY(ensure_tc_pcg(c));
  TRY(batch_alloc(c, bb, B));
  const auto t0 = std::chrono::steady_clock::now();
  const Options& o = c->opt;
  const double s_eq = c->s_equal;
  const bool stdz = o.pref_scaling == 1 && s_eq > 0.0 && isfinite(s_eq);
  const double scale = c->mu_absmax, gap_tol = o.cal_rel_tol * scale;
  const size_t ld = (size_t)c->ld;
  std::vector<InstRun> run((size_t)B);
  std::vector<std::array<double, 4>> cc((size_t)B);
  for (int b = 0; b < B; ++b) {
    InstRun& r = run[(size_t)b];
    for (int q = 0; q < 4; ++q) {
      r.lam[q] = lam_h[4 * b + q];
      r.cc[q] = stdz ? r.lam[q] / pow(s_eq, q + 1) : r.lam[q];
    }
    r.target = tg_h[b];
    cc[(size_t)b] = r.cc;
    r.c1_ref = fmax(r.cc[1], 1e-300) * s_eq * s_eq / fmax(scale, 1e-300);
    r.c1_max = 1e6 * r.c1_ref;
  }
  // device buffers for warm starts: instance scratch columns 20 (lo) and 21 (hi)
  auto xlo = [&](int b) { return inst_at(bb.base, b).tmp + (size_t)20 * ld; };
  auto xhi = [&](int b) { return inst_at(bb.base, b).tmp + (size_t)21 * ld; };
  double* w0buf = nullptr;
  if (W0 != nullptr) {
    // W0 (B x n, host or device) into each instance's bestx slot first, validated on the host
    std::vector<double> hw((size_t)B * c->n);
    CU(cudaMemcpy(hw.data(), W0, sizeof(double) * hw.size(), cudaMemcpyDefault));
    for (int b = 0; b < B; ++b) {
      double sm = 0.0, mn = INFINITY;
      for (int i = 0; i < c->n; ++i) {
        sm += hw[(size_t)b * c->n + i];
        mn = fmin(mn, hw[(size_t)b * c->n + i]);
      }
      if (!(fabs(sm - 1.0) <= 1e-9) || mn < o.tau * (1.0 - 1e-9)) return fail(MVSK_EINVAL, "W0 row %d not in Delta(tau)", b);
      CU(cudaMemsetAsync(inst_at(bb.base, b).xbar, 0, sizeof(double) * ld, c->stream));
      CU(cudaMemcpyAsync(inst_at(bb.base, b).xbar, hw.data() + (size_t)b * c->n, sizeof(double) * c->n,
                         cudaMemcpyHostToDevice, c->stream));
    }
    TRY(sync(c));
    w0buf = (double*)1;  // marker: warm starts live in each instance's xbar
  }
  // graph of one lockstep iteration (c1 is read on the device, so calibration needs no re-capture)
  cudaGraphExec_t gexec = nullptr;
  long long per_graph = 0;
  {
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const long long l0 = c->launches;
    c->ev_graph_begin = c->ev_kind.size();
    const mvsk_status cs = batch_iteration(c, bb, B, cc);
    c->ev_graph_end = c->ev_kind.size();
    per_graph = c->launches - l0;
    c->launches = l0;
    const cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
    if (cs != MVSK_OK) {
      if (g) cudaGraphDestroy(g);
      return cs;
    }
    CU(ce);
    const cudaError_t ie = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    CU(ie);
  }
  struct GraphGuard {
    cudaGraphExec_t e;
    ~GraphGuard() {
      if (e) cudaGraphExecDestroy(e);
    }
  } guard{gexec};
  // start every instance
  for (int b = 0; b < B; ++b) {
    InstRun& r = run[(size_t)b];
    const double* w0 = w0buf ? inst_at(bb.base, b).xbar : nullptr;
    if (isnan(r.target)) {
      r.cal = 0;
      TRY(batch_start_run(c, bb, b, r, r.cc[0], w0, tol));
    } else {
      r.cal = 1;
      TRY(batch_start_run(c, bb, b, r, 0.0, nullptr, tol));
    }
  }
  std::vector<int> si((size_t)B * kSI);
  std::vector<double> evh((size_t)B * 4);
  double* evd = c->vec_scratch + 64;  // not used concurrently with W0 checks (done above)
  (void)evd;
  const double phase_eta[3] = {o.eta, o.restart_eta1, o.restart_eta2};
  const int phase_it[3] = {o.pcg_max_iter, o.restart_iter, o.restart_iter};
  int remaining = B;
  const int every = 3;
  long long guard_iters = 0;
  while (remaining > 0) {
    for (int q = 0; q < every; ++q) {
      CU(cudaGraphLaunch(gexec, c->stream));
      c->launches += per_graph;
      if (c->prof_on) {
        CU(cudaStreamSynchronize(c->stream));
        TRY(prof_collect(c, c->ev_graph_begin, c->ev_graph_end));
      }
    }
    guard_iters += every;
    CU(cudaMemcpyAsync(si.data(), bb.base.si, sizeof(int) * si.size(), cudaMemcpyDeviceToHost, c->stream));
    TRY(sync(c));
    // finished inner solves: evaluate them together
    std::vector<int> fin;
    for (int b = 0; b < B; ++b) {
      InstRun& r = run[(size_t)b];
      if (r.finished) continue;
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
        k_new_phase<<<1, 32, 0, c->stream>>>(inst_at(bb.base, b), phase_eta[r.phase], phase_it[r.phase]);
        c->launches += 1;
        CU(cudaGetLastError());
        continue;
      }
      r.run_status = d2 == 1 ? MVSK_OK : (d2 == 3 ? MVSK_ENUMERIC : (d2 == 4 ? MVSK_ETIMEOUT : MVSK_ENOTCONVERGED));
      r.iters += si[(size_t)b * kSI + SI_ITER];
      const Inst s = inst_at(bb.base, b);
      if (r.run_status != MVSK_OK) CU(cudaMemcpyAsync(s.x, s.bestx, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
      fin.push_back(b);
    }
    if (fin.empty()) continue;
    for (int b : fin) {
      const Inst s = inst_at(bb.base, b);
      PassArgs a = pass_args_inst(run[(size_t)b].cc.data());
      a.in[0] = s.x;
      a.rowout = s.z;
      TRY(run_pass(c, P64, M_VALGRAD, 1, a, nullptr, s.spart));
      TRY(reduce_cols(c, P64, 1, s.g, c->ld, c->mu, 0.0, nullptr, nullptr, s.sd + SD_C1));
      k_eval_finish<<<1, kVT, 0, c->stream>>>(s, nullptr, c->grid, s.tmp + (size_t)23 * ld);
      CU(cudaMemcpyAsync(evh.data() + 4 * (size_t)b, s.tmp + (size_t)23 * ld, 3 * sizeof(double),
                         cudaMemcpyDeviceToHost, c->stream));
      CU(cudaMemcpyAsync(evh.data() + 4 * (size_t)b + 3, s.sd + SD_KKT0, sizeof(double), cudaMemcpyDeviceToHost,
                         c->stream));
      c->launches += 1;
    }
    TRY(sync(c));
    for (int b : fin) {
      InstRun& r = run[(size_t)b];
      const Inst s = inst_at(bb.base, b);
      for (int q = 0; q < 3; ++q) r.ev[q] = evh[4 * (size_t)b + q];
      const double h = r.ev[2] - r.target;
      auto finish = [&](bool from_hi) -> mvsk_status {
        if (from_hi) {
          CU(cudaMemcpyAsync(s.x, xhi(b), sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
          r.cc[0] = r.c_hi;
          r.final_from_hi = true;
        }
        r.finished = true;
        remaining -= 1;
        return MVSK_OK;
      };
      auto illinois = [&]() -> mvsk_status {
        if (r.evals >= o.cal_max_evals) return finish(true);
        double cm = r.c_hi - r.h_hi * (r.c_hi - r.c_lo) / (r.h_hi - r.h_lo);
        if (!(r.c_lo < cm && cm < r.c_hi)) cm = 0.5 * (r.c_lo + r.c_hi);
        const double* w0 = (cm - r.c_lo) <= (r.c_hi - cm) ? xlo(b) : xhi(b);
        r.cal = 3;
        return batch_start_run(c, bb, b, r, cm, w0, tol);
      };
      if (r.cal == 0) {
        TRY(finish(false));
      } else if (r.cal == 1) {
        if (h >= -gap_tol) {
          TRY(finish(false));
        } else {
          CU(cudaMemcpyAsync(xlo(b), s.x, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
          r.c_lo = 0.0;
          r.h_lo = h;
          r.c_hi = r.lam[0] > 0.0 ? (stdz ? r.lam[0] / s_eq : r.lam[0]) : r.c1_ref;
          r.cal = 2;
          TRY(batch_start_run(c, bb, b, r, r.c_hi, xlo(b), tol));
        }
      } else if (r.cal == 2) {
        r.h_hi = h;
        CU(cudaMemcpyAsync(xhi(b), s.x, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
        if (h < 0.0 && r.c_hi < r.c1_max) {
          r.c_lo = r.c_hi;
          r.h_lo = r.h_hi;
          CU(cudaMemcpyAsync(xlo(b), xhi(b), sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
          r.c_hi = fmin(8.0 * r.c_hi, r.c1_max);
          TRY(batch_start_run(c, bb, b, r, r.c_hi, xlo(b), tol));
        } else if (h < 0.0 || fabs(h) <= gap_tol) {
          TRY(finish(false));
        } else {
          r.side = 0;
          TRY(illinois());
        }
      } else {
        const double cm = r.cc[0];
        if (fabs(h) <= gap_tol || (r.c_hi - r.c_lo) <= o.cal_bracket_tol * r.c_hi) {
          TRY(finish(false));
        } else {
          if (h < 0.0) {
            r.c_lo = cm;
            r.h_lo = h;
            CU(cudaMemcpyAsync(xlo(b), s.x, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
            if (r.side == -1) r.h_hi *= 0.5;
            r.side = -1;
          } else {
            r.c_hi = cm;
            r.h_hi = h;
            CU(cudaMemcpyAsync(xhi(b), s.x, sizeof(double) * ld, cudaMemcpyDeviceToDevice, c->stream));
            if (r.side == 1) r.h_lo *= 0.5;
            r.side = 1;
          }
          TRY(illinois());
        }
      }
    }
    if (guard_iters > 1000000) return fail(MVSK_ECUDA, "batched solve did not terminate");
  }
  // results
  std::vector<double> hx(ld);
  mvsk_status first = MVSK_OK;
  for (int b = 0; b < B; ++b) {
    InstRun& r = run[(size_t)b];
    const Inst s = inst_at(bb.base, b);
    if (r.final_from_hi) {  // re-evaluate at the bracket end that is returned
      PassArgs a = pass_args_inst(r.cc.data());
      double c1 = r.cc[0];
      CU(cudaMemcpyAsync(s.sd + SD_C1, &c1, sizeof(double), cudaMemcpyHostToDevice, c->stream));
      a.in[0] = s.x;
      a.rowout = s.z;
      TRY(run_pass(c, P64, M_VALGRAD, 1, a, nullptr, s.spart));
      TRY(reduce_cols(c, P64, 1, s.g, c->ld, c->mu, 0.0, nullptr, nullptr, s.sd + SD_C1));
      k_eval_finish<<<1, kVT, 0, c->stream>>>(s, nullptr, c->grid, s.tmp + (size_t)23 * ld);
      CU(cudaMemcpyAsync(r.ev, s.tmp + (size_t)23 * ld, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      TRY(sync(c));
    }
    CU(cudaMemcpyAsync(W_out + (size_t)b * c->n, s.x, sizeof(double) * c->n, cudaMemcpyDefault, c->stream));
    if (infos != nullptr) {
      CU(cudaMemcpyAsync(hx.data(), s.x, sizeof(double) * ld, cudaMemcpyDeviceToHost, c->stream));
      double k0 = 0.0;
      CU(cudaMemcpyAsync(&k0, s.sd + SD_KKT0, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      int cnt[kSI];
      CU(cudaMemcpyAsync(cnt, s.si, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
      TRY(sync(c));
      mvsk_info& inf = infos[b];
      memset(&inf, 0, sizeof(inf));
      inf.iters = r.iters;
      inf.restarts = r.restarts;
      inf.krylov_iters = cnt[SI_KRY];
      inf.third_calls = cnt[SI_THIRD];
      inf.evals = r.evals;
      inf.f = r.ev[0];
      inf.kkt_residual = r.ev[1];
      inf.kkt0 = k0;
      inf.kkt_rel = r.ev[1] / fmax(k0, 1e-300);
      for (int q = 0; q < 4; ++q) inf.c[q] = r.cc[q];
      inf.achieved_mean = r.ev[2];
      inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      inf.status = r.run_status;
      int fc = 0;
      for (int i = 0; i < c->n; ++i) fc += (hx[(size_t)i] - o.tau > o.eps_act);
      inf.free_count = fc;
    }
    if (r.run_status != MVSK_OK && first == MVSK_OK) first = (mvsk_status)r.run_status;
  }
  TRY(sync(c));
  return first;
}
