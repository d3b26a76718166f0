// Device kernels of one YAND-MVSK iteration (Alg. 1) for one instance:
// oracle-block bookkeeping, affine-normal block in the PCG configuration,
// quartic step and boundary block.  All kernels read SI_DONE (and their own
// skip flags) first, so a fixed launch sequence can run past convergence.
#pragma once

#include "vec.cuh"

namespace mvsk {

// ---------------------------------------------------------------- utilities
static __global__ void k_fill(double* v, int n, int ld, double val) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ld; i += gridDim.x * blockDim.x) v[i] = i < n ? val : 0.0;
}

// Sum of the cross-CTA scalar partials [G][ns] -> out[ns] (fixed order).
inline __device__ void reduce_spart(const double* spart, int G, int ns, double scale, double* out) {
  if (threadIdx.x < ns) {
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += spart[(size_t)b * ns + threadIdx.x];
    out[threadIdx.x] = s * scale;
  }
  __syncthreads();
}

// Column partials [G][nout][ld] -> out[m*ld + j] = scale * sum_b part + bias_scale * bias (m = 0).
// When c1p is given the bias scale is -(*c1p) (read on the device, so a
// captured graph follows changes of c1).
template <typename acc>
static __global__ void k_reduce_cols(const acc* part, int G, int nout, int ld, int n, double scale, const double* bias,
                              double bias_scale, double* out, size_t out_stride, const int* skip, const int* live,
                              const double* c1p = nullptr) {
  if (skip != nullptr && *skip != 0) return;
  if (live != nullptr && *live == 0) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (j >= ld) return;
  double s = 0.0;
  for (int b = 0; b < G; ++b) s += (double)part[((size_t)b * nout + m) * ld + j];
  s *= scale;
  if (c1p != nullptr) bias_scale = -*c1p;
  if (bias != nullptr && m == 0) s += bias_scale * bias[j];
  out[(size_t)m * out_stride + j] = j < n ? s : 0.0;
}

// P_V v on the face F: v_F - mean_F(v) - (nu^T v) nu, zero off F.
inline __device__ void project_V(const double* v, double* out, const double* maskF, const double* nuhat, int n, double m,
                          double* scr) {
  double s = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    s += maskF[i] * v[i];
    t += nuhat[i] * v[i];
  }
  const double4 r = block_sum2_fin(s, t, scr, [=](double x, double) { return make_double2(x / m, 0.0); });
  const double mean = r.z;
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = maskF[i] * (v[i] - mean) - r.y * nuhat[i];
  __syncthreads();
}

// ------------------------------------------------------------- kkt at x0
static __global__ void __launch_bounds__(kVT) k_kkt0(Inst s0) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ double scr[80];
  const double tau = s.sd[SD_TAU];
  const double k0 = kkt_residual(s.x, s.g, s.n, tau, scr, s.tmp);
  if (threadIdx.x == 0) s.sd[SD_KKT0] = k0;
}

// f = -c1 mu^T x + T^-1 sum psi(z) and the KKT residual (mvsk_eval).
static __global__ void __launch_bounds__(kVT) k_eval_finish(Inst s0, const double* spart, int G, double* out3) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ double scr[80];
  __shared__ double ps[2];
  reduce_spart(s.spart, G, 1, s.sd[SD_INVT], ps);
  double mx = 0.0;
  for (int i = threadIdx.x; i < s.n; i += blockDim.x) mx += s.mu[i] * s.x[i];
  mx = block_sum2(mx, 0.0, scr).x;
  const double k = kkt_residual(s.x, s.g, s.n, s.sd[SD_TAU], scr, s.tmp);
  if (threadIdx.x == 0) {
    out3[0] = -s.sd[SD_C1] * mx + ps[0];
    out3[1] = k;
    out3[2] = mx;
  }
}

// ----------------------------------------------------------- oracle block
// After the value/gradient pass: objective, KKT test, best iterate, stall
// test, the working face (face continuation) and the normalised face gradient.
static __global__ void __launch_bounds__(kVT) k_face(Inst s0, const double* spart, int G) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ double scr[80];
  __shared__ double ps[2];
  __shared__ int s_stop, s_better;
  __shared__ long long s_klo, s_khi;
  int* SI = s.si;
  double* SD = s.sd;
  if (SI[SI_DONE] != 0) return;
  const int n = s.n;
  const double tau = SD[SD_TAU];
  const bool dir_only = SI[SI_DIRONLY] != 0;
  reduce_spart(s.spart, G, 1, SD[SD_INVT], ps);
  double mx = 0.0, nonfin = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    mx += s.mu[i] * s.x[i];
    if (!isfinite(s.g[i])) nonfin += 1.0;
  }
  const double2 r0 = block_sum2(mx, nonfin, scr);
  if (threadIdx.x == 0) s_stop = 0;
  __syncthreads();
  if (!dir_only) {
    if (threadIdx.x == 0) {
      const double f = -SD[SD_C1] * r0.x + ps[0];
      SD[SD_F] = f;
      SD[SD_MUX] = r0.x;
      if (r0.y > 0.0 || !isfinite(f)) {
        SI[SI_DONE] = 3;
        s_stop = 1;
      } else if (SI[SI_PHASEIT] >= SI[SI_MAXIT]) {
        SI[SI_DONE] = 2;
        s_stop = 1;
      }
      if (s_stop) {
        SI[SI_SKIPDIR] = 1;
        SI[SI_SKIPLS] = 1;
      }
    }
    __syncthreads();
    if (s_stop) return;
    const double2 kr = kkt_residual_rel(s.x, s.g, n, tau, scr, s.tmp, SD[SD_KKT0]);
    const double kkt = kr.x, rel = kr.y;
    if (threadIdx.x == 0) {
      const bool better = rel < SD[SD_BEST];
      s_better = better;
      SD[SD_KKT] = kkt;
      SD[SD_KKTREL] = rel;
      if (better) SD[SD_BEST] = rel;
      const int hn = SI[SI_HISTN];
      SD[SD_HIST + (hn & 15)] = rel;
      SI[SI_HISTN] = hn + 1;
      const int win = SI[SI_STALLWIN];
      if (rel <= SD[SD_TOL]) {
        SI[SI_DONE] = 1;
        s_stop = 1;
      } else if (SI[SI_PCG] && hn + 1 > win && win > 0 && win < 16 &&
                 rel > SD[SD_STALLF] * SD[SD_HIST + ((hn - win) & 15)]) {
        SI[SI_DONE] = 2;
        s_stop = 1;
      }
      if (s_stop) {
        SI[SI_SKIPDIR] = 1;
        SI[SI_SKIPLS] = 1;
      }
    }
    __syncthreads();
    if (s_better)
      for (int i = threadIdx.x; i < n; i += blockDim.x) s.bestx[i] = s.x[i];
    if (s_stop) return;
  }
  // Working face: coordinates at tau are held, except every one whose
  // violation nu_F - g_i is at least ||gbar_F|| / release_ratio.  Coordinate
  // i = threadIdx.x + e kVT (n <= kSliceE kVT) is held in registers; bit e of
  // fr / mf marks it above tau / on the face, so that the FP64 arithmetic
  // runs on the face's coordinates only.
  const double eps = SD[SD_EPSACT];
  double gv[kSliceE];
  unsigned fr = 0;
  double sg = 0.0;
  int cf = 0;
#pragma unroll
  for (int e = 0; e < kSliceE; ++e) {
    const int i = threadIdx.x + e * kVT;
    gv[e] = 0.0;
    if (i < n) {
      gv[e] = s.g[i];
      const double xi = s.x[i];
      if (!same_bits(xi, tau) && xi - tau > eps) {  // x = tau: 0 <= eps
        fr |= 1u << e;
        sg += gv[e];
        cf += 1;
      }
    }
  }
  const Sum2c r1 = block_sum2c_fin(sg, 0.0, cf, scr, [](double x, double, int k) { return make_double2(x / k, 0.0); });
  double nuF = r1.z;
  const int free0 = r1.k;  // coordinates above tau
  double gq = 0.0;
#pragma unroll
  for (int e = 0; e < kSliceE; ++e)
    if ((fr >> e) & 1u) {
      const double d = gv[e] - nuF;
      gq += d * d;
    }
  const double rr = SD[SD_RELRATIO];
  // The release test v = nuF - g_i > 0 and gn0 <= rr v holds for g_i below
  // T = nuF - gn0 / rr and fails above it; integer keys of T -+ delta (delta
  // far above the rounding of either form) settle all but a narrow band,
  // which takes the FP64 test itself.  (INT64_MIN: no screening.)
  long long* pklo = &s_klo;
  long long* pkhi = &s_khi;
  const double gn0 = block_sum2_fin(gq, 0.0, scr, [=](double x, double) {
                       const double g0 = sqrt(x);
                       long long lo = INT64_MIN, hi = INT64_MIN;
                       if (rr > 0.0 && g0 >= 0.0 && isfinite(rr) && isfinite(g0) && isfinite(nuF)) {
                         const double q = g0 / rr, T = nuF - q, dl = 1e-9 * (fabs(nuF) + q + fabs(T)) + 1e-300;
                         lo = dkey(T - dl);
                         hi = dkey(T + dl);
                       }
                       *pklo = lo;
                       *pkhi = hi;
                       return make_double2(g0, 0.0);
                     }).z;
  const long long klo = s_klo, khi = s_khi;
  unsigned mf = fr;
  sg = 0.0;
  int cm = 0;
#pragma unroll
  for (int e = 0; e < kSliceE; ++e) {
    const int i = threadIdx.x + e * kVT;
    if (i < n) {
      if (!((fr >> e) & 1u)) {
        const long long kg = dkey(gv[e]);
        const bool fin = ((__double_as_longlong(gv[e]) >> 52) & 0x7FF) != 0x7FF;
        bool rel;
        if (fin && kg < klo) {
          rel = true;
        } else if (fin && kg > khi && khi != INT64_MIN) {
          rel = false;
        } else {
          const double v = nuF - gv[e];
          rel = v > 0.0 && gn0 <= rr * v;
        }
        if (rel) mf |= 1u << e;
      }
      const bool on = (mf >> e) & 1u;
      s.maskF[i] = on ? 1.0 : 0.0;
      if (on) {
        sg += gv[e];
        cm += 1;
      }
    }
  }
  const Sum2c r = block_sum2c_fin(sg, 0.0, cm, scr, [](double x, double, int k) { return make_double2(x / k, 0.0); });
  const int mi = r.k;
  nuF = r.z;
  // gbar = P_F g, centred twice: the second pass removes the rounding of the
  // first relative to gbar itself (not to g), so 1_F^T nu stays at rounding
  // level even when ||gbar|| << |g| near a stationary point.
  double sb = 0.0;
#pragma unroll
  for (int e = 0; e < kSliceE; ++e) {
    gv[e] = ((mf >> e) & 1u) ? gv[e] - nuF : 0.0;
    sb += gv[e];
  }
  const double mb = block_sum2_fin(sb, 0.0, scr, [=](double x, double) { return make_double2(x / (double)mi, 0.0); }).z;
  gq = 0.0;
#pragma unroll
  for (int e = 0; e < kSliceE; ++e)
    if ((mf >> e) & 1u) {
      gv[e] -= mb;
      gq += gv[e] * gv[e];
    }
  const double4 rg = block_sum2_fin(gq, 0.0, scr, [](double x, double) {
    const double v = sqrt(x);
    return make_double2(v, v > 0.0 ? 1.0 / v : 0.0);
  });
  const double gn = rg.z, inv_gn = rg.w;  // one FP64 division instead of n
  const bool gpos = !is_zero_bits(inv_gn);   // gn > 0 (inv_gn is 0 otherwise)
  const bool trivial = mi <= 2 || !gpos;
#pragma unroll
  for (int e = 0; e < kSliceE; ++e) {
    const int i = threadIdx.x + e * kVT;
    if (i < n) {
      const double nh = (((mf >> e) & 1u) && gpos) ? gv[e] * inv_gn : 0.0;
      s.nuhat[i] = nh;
      if (trivial) s.d[i] = (mi == 2) ? -nh : 0.0;
    }
  }
  for (int i = n + threadIdx.x; i < s.ld; i += kVT) {
    s.nuhat[i] = 0.0;
    if (trivial) s.d[i] = 0.0;
  }
  if (threadIdx.x == 0) {
    SD[SD_GN] = gn;
    SD[SD_NUF] = nuF;
    SI[SI_M] = mi;
    SI[SI_SKIPDIR] = trivial ? 1 : 0;
    SI[SI_NREL] += mi - free0;  // coordinates released this iteration
  }
}

// --------------------------------------------------- PCG configuration
// Column layout: 0 = h (Newton part), 1..K = Hutchinson probes, K+1 = a.
//
// Krylov vectors X, R, Z, P, Q and the right-hand sides Bv hold elements of
// type KT: double for single-instance solves, float for lockstep batches
// (their operator products are BF16 tensor-core products, so FP32 recurrences
// lose nothing; the FP64 pipe of this part is ~2 FMA/clk/SM).  Face data in KT:
// for double the instance's own arrays, for float the copies in s.kf
// ([maskF | nuhat | diag G] written by k_pcg_setup).  Dot products are
// accumulated per thread in KT and reduced across the block in double.
template <typename KT>
struct Face {
  const KT* mf;
  const KT* nh;
  const KT* dg;
};
template <typename KT>
__device__ __forceinline__ Face<KT> face_of(const Inst& s);
template <>
__device__ __forceinline__ Face<double> face_of<double>(const Inst& s) {
  return {s.maskF, s.nuhat, s.diagG};
}
template <>
__device__ __forceinline__ Face<float> face_of<float>(const Inst& s) {
  return {s.kf, s.kf + s.ld, s.kf + 2 * (size_t)s.ld};
}
template <typename KT>
__device__ __forceinline__ KT* kcol(double* base, int c, int ld) {
  return reinterpret_cast<KT*>(base) + (size_t)c * ld;
}

// P_V v on the face (see project_V), v of type TI, out and face data of type KT.
template <typename KT, typename TI>
inline __device__ void project_Vk(const TI* v, KT* out, const Face<KT>& f, int n, double m, double* scr) {
  KT a = 0, b = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a += f.mf[i] * (KT)v[i];
    b += f.nh[i] * (KT)v[i];
  }
  const double4 r = block_sum2_fin((double)a, (double)b, scr, [=](double x, double) { return make_double2(x / m, 0.0); });
  const KT mean = (KT)r.z, ny = (KT)r.y;
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = f.mf[i] * ((KT)v[i] - mean) - ny * f.nh[i];
  __syncthreads();
}

template <typename KT>
inline __device__ void pcg_init_col(Inst& s, int c, double m, double* scr) {
  const int n = s.n, ld = s.ld;
  const Face<KT> f = face_of<KT>(s);
  KT* X = kcol<KT>(s.X, c, ld);
  KT* R = kcol<KT>(s.R, c, ld);
  KT* Z = kcol<KT>(s.Zc, c, ld);
  KT* P = kcol<KT>(s.P, c, ld);
  const KT* B = kcol<KT>(s.Bv, c, ld);
  KT* tk = reinterpret_cast<KT*>(s.tmp);
  KT nb = 0;
  for (int i = threadIdx.x; i < ld; i += blockDim.x) {
    X[i] = 0;
    R[i] = B[i];
    tk[i] = i < n ? B[i] / f.dg[i] : (KT)0;
    nb += B[i] * B[i];
  }
  __syncthreads();
  project_Vk<KT, KT>(tk, Z, f, n, m, scr);
  KT rz = 0;
  for (int i = threadIdx.x; i < ld; i += blockDim.x) {
    P[i] = Z[i];
    rz += R[i] * Z[i];
  }
  const double2 r = block_sum2((double)rz, (double)nb, scr);
  if (threadIdx.x == 0) {
    s.rz[c] = r.x;
    s.rhsn[c] = sqrt(r.y);  // one thread
    s.si[SI_ACT + c] = r.y > 0.0 ? 1 : 0;
    s.si[SI_CITS + c] = 0;
  }
  __syncthreads();
}

// Setup of the first PCG round: lambda, Jacobi diagonal, RHS h and probes.
template <typename KT>
static __global__ void __launch_bounds__(kVT) k_pcg_setup(Inst s0, const double* spart, int G, int ngroups) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ double scr[80];
  __shared__ double ps[2];
  int* SI = s.si;
  double* SD = s.sd;
  if (SI[SI_DONE] != 0 || SI[SI_SKIPDIR] != 0) return;
  const int n = s.n, ld = s.ld;
  const double m = (double)SI[SI_M];
  reduce_spart(s.spart, G, 2, SD[SD_INVT], ps);  // nu^T G nu, 1_F^T G 1_F
  // |diag G| floored, on F; 1 off F (never used there: vectors vanish off F).
  double sd = 0.0, sa = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sd += s.maskF[i] * s.diagG[i];
    sa += s.maskF[i] * fabs(s.diagG[i]);
  }
  const double psum1 = ps[1], psum0 = ps[0], reg = SD[SD_REG];
  const double4 r = block_sum2_fin(sd, sa, scr, [=](double x, double y) {
    const double trG = x - psum1 / m - psum0;
    return make_double2(1e-300 + 1e-12 * (y / m), reg * fabs(trG) / (m - 2.0));
  });
  const double floor_ = r.z, lam = r.w;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    s.diagG[i] = s.maskF[i] != 0.0 ? fmax(fabs(s.diagG[i]), floor_) : 1.0;
  if constexpr (sizeof(KT) == sizeof(float)) {
    for (int i = threadIdx.x; i < ld; i += blockDim.x) {
      s.kf[i] = i < n ? (float)s.maskF[i] : 0.f;
      s.kf[ld + i] = i < n ? (float)s.nuhat[i] : 0.f;
      s.kf[2 * (size_t)ld + i] = i < n ? (float)s.diagG[i] : 1.f;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) SD[SD_LAM] = lam;
  if (ngroups < 0) return;  // the columns are set up by k_pcg_setup_cols
  const Face<KT> f = face_of<KT>(s);
  // RHS 0: h = P_V (G nu)
  project_Vk<KT, double>(s.Gnu, kcol<KT>(s.Bv, 0, ld), f, n, m, scr);
  const int K = SI[SI_PROBES];
  for (int k = 0; k < K; ++k) project_Vk<KT, KT>(kcol<KT>(s.Bv, k + 1, ld), kcol<KT>(s.Bv, k + 1, ld), f, n, m, scr);
  for (int c = 0; c <= K; ++c) pcg_init_col<KT>(s, c, m, scr);
  if (threadIdx.x == 0) {
    for (int g = 0; g < ngroups; ++g) {
      int live = 0;
      for (int c = 2 * g; c < 2 * g + 2 && c <= K; ++c) live += SI[SI_ACT + c];
      SI[SI_LIVE + g] = live;
    }
  }
}

// Column c = blockIdx.x of the first PCG round of instance blockIdx.y, after
// k_pcg_setup(..., ngroups = -1): right-hand side (h = P_V G nu for c = 0, the
// projected probe otherwise) and the PCG start.  Scratch: the instance's tmp
// column 2 + c.  SI_LIVE is not used by the batched steps.
template <typename KT>
static __global__ void __launch_bounds__(512) k_pcg_setup_cols(Inst s0) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ double scr[80];
  int* SI = s.si;
  if (SI[SI_DONE] != 0 || SI[SI_SKIPDIR] != 0) return;
  const int c = blockIdx.x;
  if (c > SI[SI_PROBES]) return;
  const int n = s.n, ld = s.ld;
  const double m = (double)SI[SI_M];
  const Face<KT> f = face_of<KT>(s);
  if (c == 0) project_Vk<KT, double>(s.Gnu, kcol<KT>(s.Bv, 0, ld), f, n, m, scr);
  else project_Vk<KT, KT>(kcol<KT>(s.Bv, c, ld), kcol<KT>(s.Bv, c, ld), f, n, m, scr);
  Inst sc = s;
  sc.tmp = s.tmp + (size_t)(2 + c) * ld;  // per-column scratch
  pcg_init_col<KT>(sc, c, m, scr);
}

// Standard normal probes zeta_k (raw, before projection) into PCG right-hand
// sides 1..K; the iteration index comes from the device state.
template <typename KT>
static __global__ void k_probe_fill(Inst s0, int K) {
  Inst s = inst_at(s0, blockIdx.z);
  if (s.si[SI_DONE] != 0 || s.si[SI_SKIPDIR] != 0) return;
  const int k = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K || i >= s.ld) return;
  const unsigned long long seed =
      ((unsigned long long)(unsigned)s.si[SI_SEEDHI] << 32) | (unsigned long long)(unsigned)s.si[SI_SEEDLO];
  KT v = 0;
  if (i < s.n) {
    if constexpr (sizeof(KT) == sizeof(float)) v = probe_value_f(seed, s.si[SI_ITER], k, i);
    else v = probe_value(seed, s.si[SI_ITER], k, i);
  }
  kcol<KT>(s.Bv, k + 1, s.ld)[i] = v;
}

// One PCG step on column blockIdx.x + c0 (Q holds G P from the products):
// q = P_V Q + lambda P, alpha = rz / p^T q, X += alpha P, R -= alpha q,
// Z = P_V (R / |diag G|), P = Z + beta P.  Each thread keeps its <= kPE
// coordinates in registers; five fused block reductions.
constexpr int kPT = 512;                          // threads per PCG column CTA
constexpr int kPE = (kMaxCols + kPT - 1) / kPT;   // coordinates per thread
// Batched form (kp.part != null): Q is taken as kp.scale * sum of the kp.splits
// FP32 split partials of the product (row b*nc + blockIdx.x), and the new P is
// also written in BF16 to kp.P16 (same row) for the next product.
struct KPart {
  const float* part;
  int splits, N, nc;
  long long ldp;
  float scale;
  __nv_bfloat16* P16;
  // face-restricted products (nullable): runtime split count rts[2], and the
  // row of coordinate i in the partials and in P16, upos[i] (< 0: none)
  const int* rts = nullptr;
  const int* upos = nullptr;
  // with uidx: the step runs over the union U only (uidx[j], j < uinfo[0]),
  // whose position j is the partial and P16 row (every Krylov vector is zero
  // off its instance's face, a subset of U)
  const int* uidx = nullptr;
  const int* uinfo = nullptr;
};

template <typename KT>
static __global__ void __launch_bounds__(kPT, sizeof(KT) == sizeof(float) ? 2 : 1)
    k_pcg_step(Inst s0, int c0, int kmaxit, KPart kp = KPart{}) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ double scr[80];
  int* SI = s.si;
  if (SI[SI_DONE] != 0 || SI[SI_SKIPDIR] != 0) return;
  const int c = c0 + blockIdx.x;
  if (SI[SI_ACT + c] == 0) return;
  const int n = s.n, ld = s.ld;
  const KT m = (KT)SI[SI_M];
  const KT lam = (KT)s.sd[SD_LAM];
  KT* X = kcol<KT>(s.X, c, ld);
  KT* R = kcol<KT>(s.R, c, ld);
  KT* Z = kcol<KT>(s.Zc, c, ld);
  KT* P = kcol<KT>(s.P, c, ld);
  const KT* Q = kcol<KT>(s.Q, c, ld);
  const Face<KT> f = face_of<KT>(s);
  KT q[kPE], p[kPE];
  KT a1 = 0, a2 = 0;
  const size_t prow = (size_t)blockIdx.y * kp.nc + blockIdx.x;
#pragma unroll
  for (int e = 0; e < kPE; ++e) {
    const int i = threadIdx.x + e * kPT;
    const bool in = i < n;
    if (kp.part != nullptr) {
      float acc = 0.f;
      if (in)
        for (int z = 0; z < kp.splits; ++z) acc += kp.part[((size_t)z * kp.N + prow) * kp.ldp + i];
      q[e] = (KT)(kp.scale * acc);
    } else {
      q[e] = in ? Q[i] : (KT)0;
    }
    p[e] = in ? P[i] : (KT)0;
    if (in) {
      a1 += f.mf[i] * q[e];
      a2 += f.nh[i] * q[e];
    }
  }
  block_sum2k<KT>(a1, a2, scr);
  KT pq = 0, unused = 0;
  const KT qmean = a1 / m;
#pragma unroll
  for (int e = 0; e < kPE; ++e) {
    const int i = threadIdx.x + e * kPT;
    if (i < n) q[e] = f.mf[i] * (q[e] - qmean) - a2 * f.nh[i] + lam * p[e];
    pq += p[e] * q[e];
  }
  block_sum2k<KT>(pq, unused, scr);
  auto deactivate = [&]() {
    if (threadIdx.x == 0) {
      SI[SI_ACT + c] = 0;
      atomicSub(&SI[SI_LIVE + c / 2], 1);
    }
  };
  if (!(pq > (KT)0)) {
    deactivate();
    return;
  }
  const KT al = (KT)s.rz[c] / pq;
  KT rv[kPE];
  KT rr = 0, b1 = 0, b2 = 0;
#pragma unroll
  for (int e = 0; e < kPE; ++e) {
    const int i = threadIdx.x + e * kPT;
    rv[e] = 0;
    if (i < n) {
      X[i] += al * p[e];
      rv[e] = R[i] - al * q[e];
      R[i] = rv[e];
      rr += rv[e] * rv[e];
      q[e] = rv[e] / f.dg[i];  // q now holds t = R / |diag G|
      b1 += f.mf[i] * q[e];
      b2 += f.nh[i] * q[e];
    } else {
      q[e] = 0;
    }
  }
  block_sum2k<KT>(rr, b1, scr);
  block_sum2k<KT>(b2, unused, scr);
  if (threadIdx.x == 0) {
    SI[SI_CITS + c] += 1;
    atomicAdd(&SI[SI_KRY], 1);
  }
  if (sqrt((double)rr) <= s.sd[SD_KTOL] * s.rhsn[c]) {
    deactivate();
    return;
  }
  const KT tmean = b1 / m;
  KT rzn = 0;
#pragma unroll
  for (int e = 0; e < kPE; ++e) {
    const int i = threadIdx.x + e * kPT;
    if (i < n) q[e] = f.mf[i] * (q[e] - tmean) - b2 * f.nh[i];
    rzn += rv[e] * q[e];
  }
  block_sum2k<KT>(rzn, unused, scr);
  const KT beta = rzn / (KT)s.rz[c];
#pragma unroll
  for (int e = 0; e < kPE; ++e) {
    const int i = threadIdx.x + e * kPT;
    if (i < n) {
      Z[i] = q[e];
      const KT pn = q[e] + beta * p[e];
      P[i] = pn;
      if (kp.P16 != nullptr) kp.P16[prow * ld + i] = __float2bfloat16((float)pn);
    }
  }
  if (threadIdx.x == 0) {
    s.rz[c] = (double)rzn;
    if (SI[SI_CITS + c] >= kmaxit) {
      SI[SI_ACT + c] = 0;
      atomicSub(&SI[SI_LIVE + c / 2], 1);
    }
  }
}

// Block sums of N floats in a fixed order (warp shuffles, then warp 0 over the
// warp partials); scr holds >= 33 * N floats.  Every thread gets the totals.
template <int N>
__device__ __forceinline__ void block_sumNf(float (&v)[N], float* scr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < N; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < N; ++q) scr[warp * N + q] = v[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      float t = lane < nw ? scr[lane * N + q] : 0.f;
      t = warp_sum(t);
      if (lane == 0) scr[32 * N + q] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < N; ++q) v[q] = scr[32 * N + q];
}

// The batched FP32 PCG step (same recurrence as k_pcg_step with kp.part set)
// with two reductions instead of five: p^T q and the new r^T z are expanded
// into sums over the stored vectors,
//   p^T q   = sum p mf Q - qmean sum p mf - (nu^T Q) sum p nu + lam sum p^2,
//   r'^T z' = sum r' mf t - tmean sum r' mf - (nu^T t) sum r' nu,  t = r' / diag,
// so that each reduction carries every sum of its phase.
//
// Launch forms: k_pcg_step_f, one CTA of 1024 threads per (instance, column)
// (grid (ncol, B)), for the K + 1 columns of the first round; k_pcg_step_fc,
// a cluster of kPCL CTAs of 512 threads per (instance, column) (grid
// (ncol * kPCL, B)), for the single correction column of the second round.
// CTA rank r of a cluster owns coordinates [r * ch, (r + 1) * ch), each thread
// kPEF1 or kPEF4 of them, every operand loaded before its first use.  The six sums of a
// phase are reduced in each CTA, written to every CTA of the cluster
// (distributed shared memory) and added there in rank order, so that all CTAs
// take the same decisions from the same totals.  One SM per instance made the
// 64 single-column steps latency-bound; spread over four SMs they take ~30 %
// less time, while the 576-CTA first-round steps lose more to the extra waves
// of cluster-wide barriers than they gain.
constexpr int kPCL = 4;
constexpr int kPEF1 = (kMaxCols + 1023) / 1024, kPEF4 = (kMaxCols + kPCL * 512 - 1) / (kPCL * 512);

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// store v to the same shared-memory word of CTA `rank` of this cluster
__device__ __forceinline__ void st_cluster_f32(float* local, uint32_t rank, float v) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
}

// Sums of six floats over the CTA (CL = 1) or the cluster: block sums, then
// exchange and rank-ordered adds.  slot: this phase's [CL][6] exchange area
// (one per phase: a fast CTA may write the next phase's sums while a slow one
// still reads this phase's).
template <int CL>
__device__ __forceinline__ void group_sum6(float (&v)[6], float* scr, float* slot, uint32_t rank) {
  block_sumNf<6>(v, scr);
  if constexpr (CL > 1) {
    if (threadIdx.x < CL * 6) {
      const uint32_t dst = threadIdx.x / 6;
      const int q = threadIdx.x - 6 * (int)dst;
      st_cluster_f32(slot + rank * 6 + q, dst, v[q]);
    }
    cluster_sync();
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      float t = 0.f;
#pragma unroll
      for (int r = 0; r < CL; ++r) t += slot[r * 6 + q];
      v[q] = t;
    }
  }
}

template <int CL, int NT, int PE>
__device__ __forceinline__ void pcg_step_body(Inst s0, int c0, int kmaxit, const KPart& kp, uint32_t rank) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ float scr[33 * 6 + 8];
  __shared__ float slot1[CL * 6], slot2[CL * 6];
  int* SI = s.si;
  // every CTA of a cluster reads the flags before any of them can change
  // them (writes follow the first cluster barrier), so all take one branch
  if (SI[SI_DONE] != 0 || SI[SI_SKIPDIR] != 0) return;
  const int col = (int)(blockIdx.x / CL), c = c0 + col;
  if (SI[SI_ACT + c] == 0) return;
  const int ld = s.ld;
  const int* __restrict__ uidx = kp.uidx;
  const int n = uidx != nullptr ? kp.uinfo[0] : s.n;  // positions covered: U, or every coordinate
  const int ch = (n + CL - 1) / CL, i0 = (int)rank * ch, i1 = i0 + ch < n ? i0 + ch : n;
  const float m = (float)SI[SI_M];
  const float lam = (float)s.sd[SD_LAM];
  const double rz_old = s.rz[c];
  // distinct arrays: restrict lets the loads of later coordinates move above
  // the stores of earlier ones
  float* __restrict__ X = kcol<float>(s.X, c, ld);
  float* __restrict__ R = kcol<float>(s.R, c, ld);
  float* __restrict__ P = kcol<float>(s.P, c, ld);
  __nv_bfloat16* __restrict__ P16 = kp.P16;
  const Face<float> f0 = face_of<float>(s);
  const float* __restrict__ fmf = f0.mf;
  const float* __restrict__ fnh = f0.nh;
  const float* __restrict__ fdg = f0.dg;
  const size_t prow = (size_t)blockIdx.y * kp.nc + col;
  float q[PE], p[PE], r[PE], xv[PE], mf[PE], nh[PE], dg[PE];
  int ci[PE];  // coordinate of each element (-1: none)
  float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // mf.Q, nu.Q, p.mf.Q, p.mf, p.nu, p.p
#pragma unroll
  for (int e = 0; e < PE; ++e) {
    const int jp = i0 + threadIdx.x + e * NT;
    ci[e] = jp < i1 ? (uidx != nullptr ? uidx[jp] : jp) : -1;
  }
#pragma unroll
  for (int e = 0; e < PE; ++e) {
    const int i = ci[e];
    q[e] = p[e] = r[e] = xv[e] = mf[e] = nh[e] = 0.f;
    dg[e] = 1.f;
    if (i >= 0) {
      p[e] = P[i];
      r[e] = R[i];
      xv[e] = X[i];
      mf[e] = fmf[i];
      nh[e] = fnh[i];
      dg[e] = fdg[i];
    }
  }
  // split-K partials: two splits' loads in flight per batch (a split loop
  // inside the coordinate loop made each coordinate a separate round trip)
  const size_t zstride = (size_t)kp.N * kp.ldp;
  const float* __restrict__ pz = kp.part + prow * kp.ldp;
  const int nspl = kp.rts != nullptr ? kp.rts[2] : kp.splits;
  const int* __restrict__ upos = kp.upos;
  int row[PE];
#pragma unroll
  for (int e = 0; e < PE; ++e) {
    const int jp = i0 + threadIdx.x + e * NT;
    row[e] = jp < i1 ? (uidx != nullptr ? jp : (upos != nullptr ? upos[ci[e]] : jp)) : -1;
  }
  int z = 0;
  for (; z + 2 <= nspl; z += 2, pz += 2 * zstride)
#pragma unroll
    for (int e = 0; e < PE; ++e)
      if (row[e] >= 0) q[e] += pz[row[e]] + pz[zstride + row[e]];
  for (; z < nspl; ++z, pz += zstride)
#pragma unroll
    for (int e = 0; e < PE; ++e)
      if (row[e] >= 0) q[e] += pz[row[e]];
#pragma unroll
  for (int e = 0; e < PE; ++e) {
    q[e] *= kp.scale;
    const float mq = mf[e] * q[e];
    a[0] += mq;
    a[1] += nh[e] * q[e];
    a[2] += p[e] * mq;
    a[3] += p[e] * mf[e];
    a[4] += p[e] * nh[e];
    a[5] += p[e] * p[e];
  }
  group_sum6<CL>(a, scr, slot1, rank);
  const float qmean = a[0] / m, ry = a[1];
  const float pq = a[2] - qmean * a[3] - ry * a[4] + lam * a[5];
  const bool lead = rank == 0 && threadIdx.x == 0;
  if (!(pq > 0.f)) {
    if (lead) {
      SI[SI_ACT + c] = 0;
      atomicSub(&SI[SI_LIVE + c / 2], 1);
    }
    return;
  }
  const float al = (float)rz_old / pq;
  float b[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // r.r, mf.t, nu.t, r.mf.t, r.mf, r.nu
#pragma unroll
  for (int e = 0; e < PE; ++e) {
    const int i = ci[e];
    if (i >= 0) {
      const float qq = mf[e] * (q[e] - qmean) - ry * nh[e] + lam * p[e];
      X[i] = xv[e] + al * p[e];
      const float rv = r[e] - al * qq;
      R[i] = rv;
      r[e] = rv;
      const float t = rv / dg[e];
      q[e] = t;  // q now holds t = R / |diag G|
      b[0] += rv * rv;
      b[1] += mf[e] * t;
      b[2] += nh[e] * t;
      b[3] += rv * mf[e] * t;
      b[4] += rv * mf[e];
      b[5] += rv * nh[e];
    }
  }
  group_sum6<CL>(b, scr, slot2, rank);
  if (lead) {
    SI[SI_CITS + c] += 1;
    atomicAdd(&SI[SI_KRY], 1);
  }
  if (sqrt((double)b[0]) <= s.sd[SD_KTOL] * s.rhsn[c]) {
    if (lead) {
      SI[SI_ACT + c] = 0;
      atomicSub(&SI[SI_LIVE + c / 2], 1);
    }
    return;
  }
  const float tmean = b[1] / m, tb2 = b[2];
  const float rzn = b[3] - tmean * b[4] - tb2 * b[5];
  const float beta = rzn / (float)rz_old;
#pragma unroll
  for (int e = 0; e < PE; ++e) {
    const int i = ci[e];
    if (i >= 0) {
      const float zz = mf[e] * (q[e] - tmean) - tb2 * nh[e];
      const float pn = zz + beta * p[e];
      P[i] = pn;
      if (row[e] >= 0) P16[prow * ld + row[e]] = __float2bfloat16(pn);
    }
  }
  if (lead) {
    s.rz[c] = (double)rzn;
    if (SI[SI_CITS + c] >= kmaxit) {
      SI[SI_ACT + c] = 0;
      atomicSub(&SI[SI_LIVE + c / 2], 1);
    }
  }
}

static __global__ void __launch_bounds__(1024, 1) k_pcg_step_f(Inst s0, int c0, int kmaxit, KPart kp) {
  pcg_step_body<1, 1024, kPEF1>(s0, c0, kmaxit, kp, 0u);
}
static __global__ void __cluster_dims__(kPCL, 1, 1) __launch_bounds__(512, 2)
    k_pcg_step_fc(Inst s0, int c0, int kmaxit, KPart kp) {
  pcg_step_body<kPCL, 512, kPEF4>(s0, c0, kmaxit, kp, cluster_rank());
}

// Correction vector a = P_V (T^-1 A^T (psi''' o rhat)) and the second PCG round.
template <typename KT>
static __global__ void __launch_bounds__(kVT) k_pcg_setup2(Inst s0, int ca, int group) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ double scr[80];
  int* SI = s.si;
  if (SI[SI_DONE] != 0 || SI[SI_SKIPDIR] != 0) return;
  const double m = (double)SI[SI_M];
  project_Vk<KT, double>(s.at, kcol<KT>(s.Bv, ca, s.ld), face_of<KT>(s), s.n, m, scr);
  pcg_init_col<KT>(s, ca, m, scr);
  if (threadIdx.x == 0) {
    SI[SI_LIVE + group] = SI[SI_ACT + ca];
    SI[SI_THIRD] += 1;
  }
}

// d = X_h - (||gbar|| / m) X_a - nu  (ambient; zero off F), re-centred on F so
// that 1^T d = 0 to rounding relative to d.
template <typename KT>
static __global__ void __launch_bounds__(kVT) k_assemble(Inst s0, int ca) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ double scr[80];
  int* SI = s.si;
  if (SI[SI_DONE] != 0 || SI[SI_SKIPDIR] != 0) return;
  const double m = (double)SI[SI_M];
  __shared__ double s_coef;
  if (threadIdx.x == 0) s_coef = s.sd[SD_GN] / m;
  __syncthreads();
  const double coef = s_coef;
  const KT* Xh = kcol<KT>(s.X, 0, s.ld);
  const KT* Xa = kcol<KT>(s.X, ca, s.ld);
  double sd = 0.0;
  for (int i = threadIdx.x; i < s.ld; i += blockDim.x) {
    const double v = i < s.n ? (double)Xh[i] - coef * (double)Xa[i] - s.nuhat[i] : 0.0;
    s.d[i] = v;
    sd += v;
  }
  const double md = block_sum2_fin(sd, 0.0, scr, [=](double x, double) { return make_double2(x / m, 0.0); }).z;
  for (int i = threadIdx.x; i < s.n; i += blockDim.x) s.d[i] -= s.maskF[i] * md;
}

// ----------------------------------------------- quartic step + boundary block
inline __device__ void ls_coefficients(Inst& s, const double* spart, int G, const double* dir, double* coef, double* scr,
                                double* ps) {
  reduce_spart(spart, G, 12, s.sd[SD_INVT], ps);
  double md = 0.0;
  for (int i = threadIdx.x; i < s.n; i += blockDim.x) {
    const double di = dir[i];
    if (!is_zero_bits(di)) md += s.mu[i] * di;  // a zero term leaves the sum as it is
  }
  md = block_sum2(md, 0.0, scr).x;
  if (threadIdx.x == 0) {
    const double c1 = s.sd[SD_C1], c2 = s.sd[SD_C2], c3 = s.sd[SD_C3], c4 = s.sd[SD_C4];
    // s20 s30 s40 s11 s21 s31 s02 s12 s22 s03 s13 s04
    coef[0] = s.sd[SD_F];
    coef[1] = -c1 * md + 2.0 * c2 * ps[3] - 3.0 * c3 * ps[4] + 4.0 * c4 * ps[5];
    coef[2] = c2 * ps[6] - 3.0 * c3 * ps[7] + 6.0 * c4 * ps[8];
    coef[3] = -c3 * ps[9] + 4.0 * c4 * ps[10];
    coef[4] = c4 * ps[11];
    for (int q = 0; q < 12; ++q) s.sd[SD_LS + q] = ps[q];
    for (int q = 0; q < 5; ++q) s.sd[SD_COEF + q] = coef[q];
  }
  __syncthreads();
}

inline __device__ void take_step(Inst& s, const double* dir, double al, const double* xbar_or_null) {
  const double tau = s.sd[SD_TAU], eps = s.sd[SD_EPSACT];
  for (int i = threadIdx.x; i < s.n; i += blockDim.x) {
    double v;
    if (xbar_or_null) {
      v = xbar_or_null[i];
    } else {
      const double xi = s.x[i], di = dir[i];
      if (same_bits(xi, tau) && is_zero_bits(di)) continue;  // stays at tau
      v = xi + al * di;
    }
    if (!same_bits(v, tau) && v - tau <= eps) v = tau;
    s.x[i] = v;
  }
  __syncthreads();
}

// After the line-search pass along d: alpha_max, the damped nominal step
// eta_k, and the branch of the boundary block (App. C.3).
// upos (nullable): positions of the coordinates in the union of the working
// faces of a lockstep batch (-1 outside); SI_LS2OUT then records whether the
// segment dstep of a taken projection has entries outside it (else 1).
static __global__ void __launch_bounds__(kVT) k_decide1(Inst s0, const double* spart, int G, const int* upos) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ double scr[80];
  __shared__ double ps[16];
  __shared__ double coef[5];
  __shared__ double s_eq, s_bc;
  int* SI = s.si;
  double* SD = s.sd;
  if (SI[SI_DONE] != 0) return;
  const int n = s.n;
  const double tau = SD[SD_TAU], eta = SD[SD_ETA];
  ls_coefficients(s, s.spart, G, s.d, coef, scr, ps);
  // The exact step on [0, eta] (warp 0; read after the reductions below).
  if (threadIdx.x < 32) {
    const double v = quartic_argmin_w(coef, eta);
    if (threadIdx.x == 0) s_eq = v;
  }
  // alpha_max = min over d_i < 0 of (x_i - tau) / (-d_i), exactly rounded: FP32
  // ratios screen the candidates within 1e-5 of their minimum, and only those
  // take the FP64 division (tens of FP64-pipe operations each on this part).
  // (Ratios beyond the FP32 range count as +inf.)
  float am32 = INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = s.d[i];
    if (neg_bits(di)) am32 = fminf(am32, (float)(s.x[i] - tau) / (float)(-di));
  }
  am32 = (float)block_min((double)am32, scr);
  double am = INFINITY;
  if (am32 < INFINITY) {
    const float thr = am32 * (1.0f + 1e-5f);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double di = s.d[i];
      if (neg_bits(di) && (float)(s.x[i] - tau) / (float)(-di) <= thr) am = fmin(am, (s.x[i] - tau) / (-di));
    }
    am = block_min(am, scr);
  }
  double eta_k = fmin(eta, s_eq);
  if (threadIdx.x == 0) {
    SD[SD_AMAX] = am;
    SI[SI_SKIPLS] = 1;
  }
  if (am >= eta_k) {
    const double al = block_line_step(coef, am, SI[SI_LSRULE], &s_bc);
    take_step(s, s.d, al, nullptr);
    if (threadIdx.x == 0) {
      SD[SD_ALPHA] = al;
      SI[SI_BRANCH] = BR_RAW;
      SI[SI_BR_RAW] += 1;
    }
    return;
  }
  double gm = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) gm += s.g[i];
  gm = block_sum2_fin(gm, 0.0, scr, [=](double x, double) { return make_double2(x / n, 0.0); }).z;
  double gt = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) gt += (s.g[i] - gm) * (s.g[i] - gm);
  gt = block_sum2_fin(gt, 0.0, scr, [](double x, double) { return make_double2(sqrt(x), 0.0); }).z;
  bool descent = false;
  const int hmax = SI[SI_ARCMAX];
  const double deps = SD[SD_DESCEPS];
  double* u = s.tmp + s.ld;  // x + eta_k d - tau of the current trial (slice_theta scratch)
  double th = 0.0;
  for (int h = 0; h <= hmax; ++h) {
    double gd = 0.0, dd = 0.0;
    {
      // the trial point xb = Pi(x + eta_k d): u and its threshold in registers
      // (coordinate threadIdx.x + e kVT; n <= kSliceE kVT)
      double uu[kSliceE];
      float uf[kSliceE];
      th = slice_theta_r(s.x, s.d, eta_k, n, tau, scr, u, uu, uf);
      const float thf = (float)th;
#pragma unroll
      for (int e = 0; e < kSliceE; ++e) {
        const int i = threadIdx.x + e * kVT;
        if (i < n) {
          const int c = gt_screen(uf[e], thf);
          const bool above = c > 0 || (c < 0 && uu[e] > th);
          const double xi = s.x[i];
          if (above || !same_bits(xi, tau)) {  // else xb = x = tau: no term
            const double xb = above ? tau + (uu[e] - th) : tau;
            const double db = xb - xi;
            gd += s.g[i] * db;
            dd += db * db;
          }
        }
      }
    }
    descent = block_sum2_fin(gd, dd, scr, [=](double x, double y) {
                return make_double2(x < -deps * gt * sqrt(y) ? 1.0 : 0.0, 0.0);
              }).z != 0.0;
    if (descent || 0.5 * eta_k <= am) break;
    eta_k *= 0.5;
  }
  if (threadIdx.x == 0) SD[SD_ETAK] = eta_k;
  if (descent) {  // u and th still hold the accepted trial
    int out = 0;
    for (int i = threadIdx.x; i < s.ld; i += blockDim.x) {
      const double xb = i < n ? tau + fmax(u[i] - th, 0.0) : 0.0;
      s.xbar[i] = xb;
      const double db = i < n ? xb - s.x[i] : 0.0;
      s.dstep[i] = db;
      out |= (upos == nullptr || upos[i] < 0) && !is_zero_bits(db);
    }
    out = __syncthreads_or(out);
    if (threadIdx.x == 0) {
      SI[SI_LS2OUT] = (upos == nullptr || out) ? 1 : 0;
      SI[SI_BRANCH] = BR_SEGMENT;
      SI[SI_BR_SEG] += 1;
      SI[SI_SKIPLS] = 0;
    }
    return;
  }
  if (am > 0.0) {
    const double al = block_line_step(coef, am, SI[SI_LSRULE], &s_bc);
    take_step(s, s.d, al, nullptr);
    if (threadIdx.x == 0) {
      SD[SD_ALPHA] = al;
      SI[SI_BRANCH] = BR_CAPPED;
      SI[SI_BR_CAP] += 1;
    }
    return;
  }
  // Face hand-off: projected-gradient segment scaled to the YAND trial length.
  double dn = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dn += s.d[i] * s.d[i];
  const double sc = block_sum2_fin(dn, 0.0, scr, [=](double x, double) {
                      return make_double2(eta * sqrt(x) / fmax(gt, 1e-300), 0.0);
                    }).z;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s.tmp[i] = -s.g[i];
  __syncthreads();
  th = slice_theta(s.x, s.tmp, sc, n, tau, scr, u);
  double gd = 0.0;
  int out = 0;
  for (int i = threadIdx.x; i < s.ld; i += blockDim.x) {
    const double xb = i < n ? tau + fmax(u[i] - th, 0.0) : 0.0;
    s.xbar[i] = xb;
    const double db = i < n ? xb - s.x[i] : 0.0;
    s.dstep[i] = db;
    if (i < n) gd += s.g[i] * db;
    out |= (upos == nullptr || upos[i] < 0) && !is_zero_bits(db);
  }
  out = __syncthreads_or(out);
  gd = block_sum2(gd, 0.0, scr).x;
  if (threadIdx.x == 0) {
    SI[SI_LS2OUT] = (upos == nullptr || out) ? 1 : 0;
    SI[SI_BRANCH] = BR_FACE;
    SI[SI_BR_FACE] += 1;
    SI[SI_SKIPLS] = gd < 0.0 ? 0 : 1;
  }
}

// After the line-search pass along the segment: exact quartic on [0, 1].
static __global__ void __launch_bounds__(kVT) k_decide2(Inst s0, const double* spart, int G) {
  Inst s = inst_at(s0, blockIdx.y);
  __shared__ double scr[80];
  __shared__ double ps[16];
  __shared__ double coef[5];
  __shared__ double s_bc;
  if (s.si[SI_DONE] != 0 || s.si[SI_SKIPLS] != 0) return;
  ls_coefficients(s, s.spart, G, s.dstep, coef, scr, ps);
  const double al = block_line_step(coef, 1.0, s.si[SI_LSRULE], &s_bc);
  take_step(s, s.dstep, al, al == 1.0 ? s.xbar : nullptr);
  if (threadIdx.x == 0) s.sd[SD_ALPHA] = al;
}

static __global__ void k_end_iter(Inst s0) {
  Inst s = inst_at(s0, blockIdx.y);
  if (threadIdx.x != 0 || s.si[SI_DONE] != 0) return;
  s.si[SI_ITER] += 1;
  s.si[SI_PHASEIT] += 1;
}

}  // namespace mvsk
