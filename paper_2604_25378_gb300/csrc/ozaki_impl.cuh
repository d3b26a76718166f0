// Host side of the emulated-FP64 tensor-core products A V and A^T V
// (kernels and the splitting in ozaki.cuh).  Included by mvsk_api.cu.
#pragma once

constexpr int kKindOz = 680;  // profiler kinds: 680 = A V, 681 = A^T V

// Digit planes of A in both orientations (once per context) and the
// right-hand tensor maps for Bp vectors (Bp a multiple of 16, at most 64).
mvsk_status oz_prepare(mvsk_ctx* c, int Bp) {
  OzBuf& o = c->oz;
  if (Bp < 16 || Bp > kOzMaxB || Bp % 16 != 0) return fail(MVSK_EINVAL, "emulated product of %d vectors", Bp);
  if (o.AF == nullptr) {
    o.MpF = (c->T + kTcBM - 1) / kTcBM * kTcBM;
    o.MpB = (c->n + kTcBM - 1) / kTcBM * kTcBM;
    o.ldT = (c->T + kTcBK - 1) / kTcBK * kTcBK;
    void* p;
    TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * kOzS * (size_t)o.MpF * c->ld));
    o.AF = (__nv_bfloat16*)p;
    TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * kOzS * (size_t)o.MpB * o.ldT));
    o.AB = (__nv_bfloat16*)p;
    TRY(dalloc(c, &p, sizeof(int) * o.MpF));
    o.eF = (int*)p;
    TRY(dalloc(c, &p, sizeof(int) * o.MpB));
    o.eB = (int*)p;
    TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * kOzS * kOzMaxB * (size_t)c->ld));
    o.XF = (__nv_bfloat16*)p;
    TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * kOzS * kOzMaxB * (size_t)o.ldT));
    o.XB = (__nv_bfloat16*)p;
    TRY(dalloc(c, &p, sizeof(int) * 2 * kOzMaxB));
    o.fF = (int*)p;
    o.fB = o.fF + kOzMaxB;
    const size_t sF = (size_t)((c->ld + kOzKc - 1) / kOzKc) * o.MpF;
    const size_t sB = (size_t)((o.ldT + kOzKc - 1) / kOzKc) * o.MpB;
    TRY(dalloc(c, &p, sizeof(long long) * kOzMaxB * (sF > sB ? sF : sB)));
    o.part = (long long*)p;
    k_oz_row_exp<<<(unsigned)((o.MpF + 7) / 8), 256, 0, c->stream>>>(c->A64, c->ld, c->T, c->n, o.eF, o.MpF);
    k_oz_split_rows<<<4 * c->nsm, 256, 0, c->stream>>>(c->A64, c->ld, c->T, c->n, o.eF, o.AF, o.MpF, c->ld);
    k_oz_col_exp<<<(unsigned)(o.MpB / 32), dim3(32, 32), 0, c->stream>>>(c->A64, c->ld, c->T, c->n, o.eB, o.MpB);
    k_oz_split_cols<<<dim3((unsigned)(o.ldT / 32), (unsigned)(o.MpB / 32)), dim3(32, 8), 0, c->stream>>>(
        c->A64, c->ld, c->T, c->n, o.eB, o.AB, o.MpB, o.ldT);
    c->launches += 4;
    CU(cudaGetLastError());

  }
  if (o.bp != Bp) {
    TRY(make_tmap_bf16(&o.tmXF, o.XF, (unsigned long long)c->ld, (unsigned long long)kOzS * Bp,
                       (unsigned long long)c->ld * 2, kTcBK, (unsigned)Bp));
    TRY(make_tmap_bf16(&o.tmXB, o.XB, (unsigned long long)o.ldT, (unsigned long long)kOzS * Bp,
                       (unsigned long long)o.ldT * 2, kTcBK, (unsigned)Bp));
    o.bp = Bp;
  }
  return MVSK_OK;
}

// Digits of the B <= Bp vectors V[b*vstride + k] and the split partials of
// A V (trans = 0: K = n, M = T) or A^T V (trans = 1: K = T, M = n) in
// c->oz.part (ld = Mp).  need: device flag (nullable); at 0 the launches
// return at once (a captured graph keeps them).
mvsk_status oz_product(mvsk_ctx* c, int trans, const double* V, long long vstride, int B, int Bp, const int* need,
                       int* splits_out) {
  TRY(oz_prepare(c, Bp));
  OzBuf& o = c->oz;
  const long long K = trans ? c->T : c->n;
  const long long ldk = trans ? o.ldT : c->ld;
  const long long M = trans ? c->n : c->T;
  const long long Mp = trans ? o.MpB : o.MpF;
  int* f = trans ? o.fB : o.fF;
  const int nkb = (int)(ldk / kTcBK);
  const int slots = oz_slots(nkb);
  const long long units = Mp / kTcBM * ((nkb + 7) / 8);
  const unsigned grid = (unsigned)(units < c->nsm ? units : c->nsm);
  const __nv_bfloat16* ad = trans ? o.AB : o.AF;
  const int nkt = nkb;
  const CUtensorMap& tx = trans ? o.tmXB : o.tmXF;
  // work: BF16 tensor FLOPs issued (kOzS (kOzS + 1) / 2 digit products)
  const double flops = 2.0 * (double)Mp * (double)((ldk + kTcBK - 1) / kTcBK * kTcBK) * Bp * (kOzS * (kOzS + 1) / 2);
  const long long zn = (long long)slots * Bp * Mp;
  PROF_LAUNCH(NK_OZ_SPLIT, (k_oz_vec_split<<<dim3((unsigned)oz_split_chunks(ldk), (unsigned)Bp), 512, 0, c->stream>>>(
                               V, vstride, B, (int)K, (int)ldk, nullptr, nullptr, f, trans ? o.XB : o.XF, Bp, o.part,
                               zn, need)));
  // launches gated by a device flag (z = A x on refreshes, the projected
  // segment) have their own kind: when skipped they do no work
  TRY(prof_begin(c, need != nullptr ? kKindOz + 2 + trans : kKindOz + trans, flops));
  switch (Bp) {
    case 16:
      k_oz_gemm<16><<<grid, kOzThreads, oz_smem_bytes(16), c->stream>>>(ad, tx, Mp, M, (int)K, nkt, o.part, Mp,
                                                                         c->err, need);
      break;
    case 32:
      k_oz_gemm<32><<<grid, kOzThreads, oz_smem_bytes(32), c->stream>>>(ad, tx, Mp, M, (int)K, nkt, o.part, Mp,
                                                                         c->err, need);
      break;
    case 48:
      k_oz_gemm<48><<<grid, kOzThreads, oz_smem_bytes(48), c->stream>>>(ad, tx, Mp, M, (int)K, nkt, o.part, Mp,
                                                                         c->err, need);
      break;
    default:
      k_oz_gemm<64><<<grid, kOzThreads, oz_smem_bytes(64), c->stream>>>(ad, tx, Mp, M, (int)K, nkt, o.part, Mp,
                                                                         c->err, need);
      break;
  }
  CU(cudaGetLastError());
  TRY(prof_end(c));
  c->launches += 1;
  *splits_out = slots;
  return MVSK_OK;
}

// A V with the left operand restricted to the columns of A in a coordinate
// list (the union of the working faces of a batch): AU holds their digit
// planes (k_oz_split_rows_u, padded count info[1]); the B vectors are
// V[b*vstride + idx[j]], j < info[0] (the list), zero beyond it.  Partials in c->oz.part
// as from oz_product (ld Mp), slot count oz_slots(info[1] / 64), read by the
// finishing kernel from info.  need: device flag (nullable) as in oz_product.
mvsk_status oz_product_u(mvsk_ctx* c, const double* V, long long vstride, const int* idx, int B, int Bp,
                         const __nv_bfloat16* AU, const int* info, const int* need) {
  TRY(oz_prepare(c, Bp));
  OzBuf& o = c->oz;
  const int K = c->ld;
  // the grid and the zeroed slots cover every column; the kernel takes its
  // k-extent from info[1] (CTAs without units return)
  const int nkb = K / kTcBK;
  const long long units = o.MpF / kTcBM * ((nkb + 7) / 8);
  const unsigned grid = (unsigned)(units < c->nsm ? units : c->nsm);
  const long long zn = (long long)oz_slots(nkb) * Bp * o.MpF;
  PROF_LAUNCH(NK_OZ_SPLIT, (k_oz_vec_split<<<dim3((unsigned)oz_split_chunks(K), (unsigned)Bp), 512, 0, c->stream>>>(
                               V, vstride, B, K, c->ld, idx, info, o.fF, o.XF, Bp, o.part, zn, need)));
  // work per unit of the padded list length: 28 digit products of Mp x Bp
  TRY(prof_begin_u(c, need != nullptr ? kKindOz + 5 : kKindOz + 4,
                   2.0 * (double)o.MpF * Bp * (kOzS * (kOzS + 1) / 2)));
  switch (Bp) {
    case 16:
      k_oz_gemm<16><<<grid, kOzThreads, oz_smem_bytes(16), c->stream>>>(AU, o.tmXF, o.MpF, c->T, K, K / 64, o.part,
                                                                         o.MpF, c->err, need, info);
      break;
    case 32:
      k_oz_gemm<32><<<grid, kOzThreads, oz_smem_bytes(32), c->stream>>>(AU, o.tmXF, o.MpF, c->T, K, K / 64, o.part,
                                                                         o.MpF, c->err, need, info);
      break;
    case 48:
      k_oz_gemm<48><<<grid, kOzThreads, oz_smem_bytes(48), c->stream>>>(AU, o.tmXF, o.MpF, c->T, K, K / 64, o.part,
                                                                         o.MpF, c->err, need, info);
      break;
    default:
      k_oz_gemm<64><<<grid, kOzThreads, oz_smem_bytes(64), c->stream>>>(AU, o.tmXF, o.MpF, c->T, K, K / 64, o.part,
                                                                         o.MpF, c->err, need, info);
      break;
  }
  CU(cudaGetLastError());
  TRY(prof_end(c));
  c->launches += 1;
  return MVSK_OK;
}

int oz_bp(int B) { return (B + 15) / 16 * 16; }

// CTAs over t of the row-wise finishing kernels (at most c->grid: the scalar
// partial slots of an instance).
int oz_row_ctas(const mvsk_ctx* c) {
  const long long g = (c->T + 255) / 256;
  return (int)(g < c->grid ? g : c->grid);
}

// CTAs per instance of the line-search power sums: four rows per thread, so
// that the twelve-sum reduction of each CTA is amortised over 1024 rows.
int oz_ls_ctas(const mvsk_ctx* c) {
  const long long g = (c->T + 1023) / 1024;
  return (int)(g < c->grid ? g : c->grid);
}
