// Single-CTA kernels for the O(n) logic of each YAND-MVSK iteration: the
// projected-simplex KKT residual, the working face, PCG vector updates in the
// ambient tangent space, and the boundary block of Alg. 1 / App. C.3.
// One CTA of kVT threads holds one instance; n <= kMaxCols.
#pragma once

#include "common.cuh"

namespace mvsk {

constexpr int kVT = 1024;
constexpr int kMaxProbes = 16;  // Hutchinson probes per direction (option "probes")

// ---------------------------------------------------------------- state slots
// Per-instance scalar state (device memory): doubles sd[kSD], ints si[kSI].
enum SD : int {
  SD_F = 0, SD_KKT, SD_KKT0, SD_KKTREL, SD_BEST, SD_GN, SD_NUF, SD_LAM, SD_AMAX, SD_ETAK,
  SD_ALPHA, SD_MUX, SD_TOL, SD_ETA, SD_TAU, SD_EPSACT, SD_RELRATIO, SD_REG, SD_KTOL, SD_C1,
  SD_C2, SD_C3, SD_C4, SD_INVT, SD_DESCEPS, SD_STALLF, SD_SUMZ2,
  SD_HIST = 32,   // 16-slot ring of kkt_rel (stall test)
  SD_LS = 48,     // 12 power sums
  SD_COEF = 60,   // A0..A4
  kSD = 72
};
enum SI : int {
  SI_DONE = 0,      // 0 running, 1 converged, 2 phase over, 3 non-finite
  SI_ITER, SI_PHASEIT, SI_MAXIT, SI_M, SI_BRANCH, SI_SKIPDIR, SI_SKIPLS, SI_PCG, SI_STALLWIN,
  SI_NREL, SI_KRY, SI_NCOL, SI_PROBES, SI_SEEDLO, SI_SEEDHI, SI_HISTN, SI_KMAXIT, SI_DIRONLY,
  SI_PASSES, SI_HVPS, SI_THIRD, SI_BR_RAW, SI_BR_SEG, SI_BR_CAP, SI_BR_FACE, SI_ARCMAX,
  SI_LSRULE,        // step rule along d: 0 exact quartic, 1 Armijo backtracking on the quartic
  SI_FCNT,          // coordinates of the working face in the face list (lockstep batches)
  SI_LS2OUT,        // the step segment dstep has entries off the union of the faces (lockstep batches)
  SI_LIVE = 30,     // live-column count per PCG group (10 groups of two columns)
  SI_ACT = 40,      // per-column active flags (20 columns)
  SI_CITS = 60,     // per-column PCG iteration counts (20 columns)
  kSI = 80
};
enum Branch : int { BR_NONE = 0, BR_RAW = 1, BR_SEGMENT = 2, BR_CAPPED = 3, BR_FACE = 4 };

// Device state of one instance.  A batch of B instances stores every array
// instance-strided; inst_at(base, b) is instance b's view.
struct Inst {
  double* sd;
  int* si;
  const double* mu;
  double *x, *g, *z, *nuhat, *maskF, *d, *dstep, *xbar, *Gnu, *diagG, *at, *bestx, *rhat, *tmp;
  double *X, *R, *Zc, *P, *Q, *Bv;  // PCG columns, [ncol][ld]
  double *rz, *rhsn;
  double* spart;  // scalar partials of this instance's streaming passes
  float* kf;      // FP32 face data of FP32 Krylov recurrences [maskF | nuhat | diag G] (batches), else null
  int n, ld;
  long long T;
  long long vs, ts, cs, ps, ncs, ss;  // instance strides: ld-vectors, T-vectors, PCG blocks, scratch, per-column, partials
  long long kfs;                      // instance stride of kf
};

__host__ __device__ __forceinline__ Inst inst_at(const Inst& a, int b) {
  Inst s = a;
  if (b != 0) {
    s.sd += (size_t)b * kSD;
    s.si += (size_t)b * kSI;
    const long long v = (long long)b * a.vs;
    s.x += v; s.g += v; s.nuhat += v; s.maskF += v; s.d += v; s.dstep += v; s.xbar += v;
    s.Gnu += (long long)b * 2 * a.vs; s.diagG += (long long)b * 2 * a.vs;
    s.at += v; s.bestx += v;
    const long long t = (long long)b * a.ts;
    s.z += t; s.rhat += t;
    s.tmp += (long long)b * a.ps;
    const long long cc = (long long)b * a.cs;
    s.X += cc; s.R += cc; s.Zc += cc; s.P += cc; s.Q += cc; s.Bv += cc;
    s.rz += (long long)b * a.ncs; s.rhsn += (long long)b * a.ncs;
    s.spart += (long long)b * a.ss;
    if (s.kf != nullptr) s.kf += (long long)b * a.kfs;
  }
  return s;
}

// Block sums of two values (see red_stage: staged in shared memory, folded by
// warps 0..3 and then warp 0); scr holds >= 68 doubles, slots 64/65
// broadcast the sums.
// block_sum2_fin also evaluates fin(x, y) -> (z, w) (a division, a square
// root, a test) once, on the thread that completes the sums, and broadcasts it
// with them: an FP64 division or square root is about ten FP64-pipe
// instructions, which every warp of the block would otherwise repeat.
// Returns {x, y, z, w}.
template <typename F>
__device__ __forceinline__ double4 block_sum2_fin(double a, double b, double* scr, F fin) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* st = red_stage();
  double* s2 = red_stage2();
  __syncthreads();
  st[threadIdx.x] = a;
  st[1024 + threadIdx.x] = b;
  __syncthreads();
  if (warp < 4) {  // rows w, w + 4, ... of warp w
    double pa = 0.0, pb = 0.0;
    for (int k = warp; k < nw; k += 4) {
      pa += st[k * 32 + lane];
      pb += st[1024 + k * 32 + lane];
    }
    s2[warp * 32 + lane] = pa;
    s2[128 + warp * 32 + lane] = pb;
  }
  __syncthreads();
  if (warp == 0) {
    double ra = s2[lane], rb = s2[128 + lane];
    for (int w = 1; w < (nw < 4 ? nw : 4); ++w) {
      ra += s2[w * 32 + lane];
      rb += s2[128 + w * 32 + lane];
    }
    const double ta = warp_sum(ra), tb = warp_sum(rb);
    if (lane == 0) {
      const double2 zw = fin(ta, tb);
      scr[64] = ta;
      scr[65] = tb;
      scr[66] = zw.x;
      scr[67] = zw.y;
    }
  }
  __syncthreads();
  return make_double4(scr[64], scr[65], scr[66], scr[67]);
}

__device__ __forceinline__ double2 block_sum2(double a, double b, double* scr) {
  const double4 r = block_sum2_fin(a, b, scr, [](double, double) { return make_double2(0.0, 0.0); });
  return make_double2(r.x, r.y);
}

// The same in FP32 (scr >= 66 floats).
__device__ __forceinline__ float2 block_sum2f(float a, float b, float* scr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if (lane == 0) {
    scr[warp] = a;
    scr[32 + warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    float ta = lane < nw ? scr[lane] : 0.f, tb = lane < nw ? scr[32 + lane] : 0.f;
    ta = warp_sum(ta);
    tb = warp_sum(tb);
    if (lane == 0) {
      scr[64] = ta;
      scr[65] = tb;
    }
  }
  __syncthreads();
  return make_float2(scr[64], scr[65]);
}

// Block sums of two values of type KT; scr holds >= 66 doubles.
template <typename KT>
__device__ __forceinline__ void block_sum2k(KT& a, KT& b, double* scr) {
  if constexpr (sizeof(KT) == sizeof(float)) {
    const float2 r = block_sum2f(a, b, reinterpret_cast<float*>(scr));
    a = r.x;
    b = r.y;
  } else {
    const double2 r = block_sum2(a, b, scr);
    a = r.x;
    b = r.y;
  }
}

// FP32 block sums of three values by warp shuffles (FP32 and integer pipes
// only); scr holds >= 99 floats.  Every thread receives the sums.
__device__ __forceinline__ float3 block_sum3f(float a, float b, float c, float* scr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  __syncthreads();
  if (lane == 0) {
    scr[warp] = a;
    scr[32 + warp] = b;
    scr[64 + warp] = c;
  }
  __syncthreads();
  if (warp == 0) {
    float ta = lane < nw ? scr[lane] : 0.f, tb = lane < nw ? scr[32 + lane] : 0.f, tc = lane < nw ? scr[64 + lane] : 0.f;
    ta = warp_sum(ta);
    tb = warp_sum(tb);
    tc = warp_sum(tc);
    if (lane == 0) {
      scr[96] = ta;
      scr[97] = tb;
      scr[98] = tc;
    }
  }
  __syncthreads();
  return make_float3(scr[96], scr[97], scr[98]);
}

// Block sums of two doubles and an int count (staged like block_sum2_fin);
// fin(a, b, k) -> (z, w) runs once, on the thread completing the sums.
struct Sum2c {
  double a, b, z, w;
  int k;
};
template <typename F>
__device__ __forceinline__ Sum2c block_sum2c_fin(double a, double b, int k, double* scr, F fin) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* st = red_stage();
  int* sti = red_stage_i();
  double* s2 = red_stage2();
  int* s2i = red_stage2_i();
  __syncthreads();
  st[threadIdx.x] = a;
  st[1024 + threadIdx.x] = b;
  sti[threadIdx.x] = k;
  __syncthreads();
  if (warp < 4) {  // rows w, w + 4, ... of warp w
    double pa = 0.0, pb = 0.0;
    int pk = 0;
    for (int w = warp; w < nw; w += 4) {
      pa += st[w * 32 + lane];
      pb += st[1024 + w * 32 + lane];
      pk += sti[w * 32 + lane];
    }
    s2[warp * 32 + lane] = pa;
    s2[128 + warp * 32 + lane] = pb;
    s2i[warp * 32 + lane] = pk;
  }
  __syncthreads();
  if (warp == 0) {
    double ra = s2[lane], rb = s2[128 + lane];
    int rk = s2i[lane];
    for (int w = 1; w < (nw < 4 ? nw : 4); ++w) {
      ra += s2[w * 32 + lane];
      rb += s2[128 + w * 32 + lane];
      rk += s2i[w * 32 + lane];
    }
    const double ta = warp_sum(ra), tb = warp_sum(rb);
    const int tk = warp_sum(rk);
    if (lane == 0) {
      const double2 zw = fin(ta, tb, tk);
      scr[64] = ta;
      scr[65] = tb;
      scr[66] = zw.x;
      scr[67] = zw.y;
      scr[68] = (double)tk;
    }
  }
  __syncthreads();
  return {scr[64], scr[65], scr[66], scr[67], (int)scr[68]};
}

// Bit tests and conversions on the integer pipe.  The FP64 pipe of this part
// runs about 2 operations/clk/SM, and most coordinates of a working face sit
// at tau with a zero direction, so exact integer tests on the bits let the
// per-instance passes skip their FP64 arithmetic there.
__device__ __forceinline__ bool is_zero_bits(double v) { return (__double_as_longlong(v) << 1) == 0; }
__device__ __forceinline__ bool same_bits(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }
// v < 0 and nonzero (a negative NaN also passes; callers then see a NaN ratio)
__device__ __forceinline__ bool neg_bits(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 && (b << 1) != 0;
}
// Order-preserving integer key of a non-NaN double (-0 sorts below +0).
__device__ __forceinline__ long long dkey(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
// (float)v truncated toward zero (relative error < 2^-23; 0 below 2^-126,
// +-inf above the FP32 range, NaN kept), by integer operations: a screening
// value, not a rounding.
__device__ __forceinline__ float f32_trunc(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (unsigned)((b >> 29) & 0x7FFFFFu) | ((b << 12) != 0 ? 1u : 0u));
  const int fe = E - 896;  // FP32 biased exponent
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
}

// The double of a finite FP32 value, by integer operations (exact).
__device__ __forceinline__ double f64_from_f32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  int E = (int)((b >> 23) & 0xFF);
  unsigned long long m = b & 0x7FFFFFu;
  if (E == 0) {
    if (m == 0) return __longlong_as_double((long long)sign);
    while ((m & 0x800000u) == 0) {  // subnormal: normalise
      m <<= 1;
      --E;
    }
    m &= 0x7FFFFFu;
    ++E;
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)(E + 896) << 52) | (m << 29)));
}

// u > th decided in FP32 from uf and thf, FP32 values of u and th within a
// relative 2^-23 (f32_trunc or a rounding) or an absolute 2^-126: 1 or 0 when
// the FP32 values settle it, -1 when the FP64 compare must.  A gap of 1e-6
// (|uf| + |thf|) + 1e-30 leaves a margin of more than 5x over both errors and
// the FP32 arithmetic of the test.
__device__ __forceinline__ int gt_screen(float uf, float thf) {
  if (!(fabsf(uf) < 1e30f) || !(fabsf(thf) < 1e30f)) return -1;
  const float gap = 1e-6f * (fabsf(uf) + fabsf(thf)) + 1e-30f;
  if (uf > thf + gap) return 1;
  if (uf < thf - gap) return 0;
  return -1;
}

// Threshold theta of the projection onto Delta(tau) of v = base + s*dir
// (dir may be null): Pi(v)_i = tau + max(v_i - tau - theta, 0), i.e. the root
// of phi(theta) = sum_i max(u_i - theta, 0) - b, u = v - tau, b = 1 - n tau.
// Michelot (1986): theta_{k+1} = (sum_{u_i > theta_k} u_i - b) / #{u_i > theta_k}
// increases monotonically to the root from any theta_0 with phi(theta_0) >= 0
// (the set {u_i > theta_k} only shrinks), and stops when the set does; the
// mean start theta_0 = (sum_i u_i - b) / n always qualifies.  u (nullable)
// receives v - tau.
//
// Coordinates are held in registers (n <= kSliceE blockDim.x; larger n take
// slice_theta_mem) and the iteration runs twice: in FP32 from the mean start
// to an estimate thf, then in FP64 from theta_0 = thf - delta, delta well
// above the FP32 error, with phi(theta_0) >= 0 checked on the first FP64 step
// (else FP64 from the mean start).  Coordinates left below a threshold stay
// out (monotonicity), and FP32 screening (gt_screen) settles most compares,
// so the FP64 pipe sees about one pass over the coordinates plus the final
// set rather than one pass per iteration.
constexpr int kSliceE = (kMaxCols + kVT - 1) / kVT;

inline __device__ double slice_theta_mem(const double* base, const double* dir, double s, int n, double tau,
                                         double* scr, double* u);

// The register form (n <= kSliceE blockDim.x): uu[e], uf[e] receive u_i and
// (float)u_i of coordinate i = threadIdx.x + e blockDim.x (0 beyond n).
__device__ __forceinline__ double slice_theta_r(const double* base, const double* dir, double s, int n, double tau,
                                                double* scr, double* u, double (&uu)[kSliceE], float (&uf)[kSliceE]) {
  // Scalar FP64 arithmetic runs only on the thread that completes each
  // reduction (its fin): on this part a uniform FP64 operation executed by
  // every thread of the block costs as much as one per coordinate.
  unsigned all = 0;
  double su = 0.0;
  float sabs = 0.f;
#pragma unroll
  for (int e = 0; e < kSliceE; ++e) {
    const int i = threadIdx.x + e * blockDim.x;
    double ui = 0.0;
    if (i < n) {
      const double bi = base[i];
      // base tau with a zero direction gives u = +0 exactly (tau + s*0 = tau)
      if (!(same_bits(bi, tau) && (dir == nullptr || is_zero_bits(dir[i])))) {
        ui = (dir ? bi + s * dir[i] : bi) - tau;
        su += ui;
      }
      if (u) u[i] = ui;
      all |= 1u << e;
    }
    uu[e] = ui;
    uf[e] = f32_trunc(ui);
    sabs += fabsf(uf[e]);
  }
  const double4 r0 = block_sum2_fin(su, (double)sabs, scr, [=](double x, double y) {
    const double b = 1.0 - (double)n * tau;
    // Michelot's mean start; its FP32 value and the mean |u| as bit patterns
    const double tm = (x - b) / (double)n;
    return make_double2(tm, __longlong_as_double(((long long)__float_as_int((float)tm) << 32) |
                                                 (unsigned)__float_as_int((float)(y / (double)n))));
  });
  const double theta_mean = r0.z;
  const long long pk = __double_as_longlong(r0.w);
  // FP32 pass: an estimate of the root and the scale of its error
  float thf = __int_as_float((int)(pk >> 32));
  float scale = __int_as_float((int)(pk & 0xFFFFFFFFll));  // mean |u| over the current set
  const float bf = 1.f - (float)n * f32_trunc(tau);
  {
    unsigned in = all;
    int cnt = n;
    for (int it = 0; it < 64; ++it) {
      float sa = 0.f, sb = 0.f;
      int ka = 0;
      unsigned nin = 0;
#pragma unroll
      for (int e = 0; e < kSliceE; ++e)
        if (((in >> e) & 1u) && uf[e] > thf) {
          sa += uf[e];
          sb += fabsf(uf[e]);
          ka += 1;
          nin |= 1u << e;
        }
      in = nin;
      const float3 r = block_sum3f(sa, sb, (float)ka, reinterpret_cast<float*>(scr));
      const int k = (int)r.z;
      if (k == cnt || k == 0) break;
      cnt = k;
      thf = (r.x - bf) / r.z;
      scale = r.y / r.z;
    }
  }
  // FP64 pass from just below the estimate (start formed in FP32 and widened
  // exactly; never below the mean start, which always qualifies)
  const float t0 = thf - 1e-4f * (fabsf(thf) + scale);
  double th = theta_mean;
  if (fabsf(t0) < 1e30f) {
    const double t0d = f64_from_f32(t0);
    if (dkey(t0d) > dkey(theta_mean)) th = t0d;
  }
  unsigned in = all;
  int cnt = -1;
  bool first = true;
  for (int it = 0; it <= n + 1; ++it) {
    const float tf = f32_trunc(th);
    double sa = 0.0;
    int ka = 0;
    unsigned nin = 0;
#pragma unroll
    for (int e = 0; e < kSliceE; ++e)
      if ((in >> e) & 1u) {
        const int c = gt_screen(uf[e], tf);
        if (c > 0 || (c < 0 && uu[e] > th)) {
          sa += uu[e];
          ka += 1;
          nin |= 1u << e;
        }
      }
    const double thc = th;
    const bool fst = first;
    const Sum2c r = block_sum2c_fin(sa, 0.0, ka, scr, [=](double x, double, int k) {
      // next iterate, and on the first step of a start above the mean start
      // whether phi(th) = sum_{u > th} (u - th) - b < 0 (th above the root):
      // then w = 1 and the iteration restarts from the mean start
      const double b = 1.0 - (double)n * tau;
      const bool restart = fst && thc > theta_mean && !((x - (double)k * thc - b) >= 0.0);
      return make_double2(k > 0 ? (x - b) / (double)k : 0.0, restart ? 1.0 : 0.0);
    });
    if (first) {
      first = false;
      if (!is_zero_bits(r.w)) {
        th = theta_mean;
        in = all;
        first = true;
        continue;
      }
    }
    if (r.k == cnt || r.k == 0) break;
    cnt = r.k;
    th = r.z;
    in = nin;
  }
  return th;
}

inline __device__ double slice_theta(const double* base, const double* dir, double s, int n, double tau, double* scr,
                                     double* u = nullptr) {
  if (n > kSliceE * (int)blockDim.x) return slice_theta_mem(base, dir, s, n, tau, scr, u);
  double uu[kSliceE];
  float uf[kSliceE];
  return slice_theta_r(base, dir, s, n, tau, scr, u, uu, uf);
}

// The same with the coordinates in memory (any n): plain FP64 Michelot from
// the mean start, u formed once into the scratch vector when one is given.
inline __device__ double slice_theta_mem(const double* base, const double* dir, double s, int n, double tau,
                                         double* scr, double* u) {
  const double b = 1.0 - (double)n * tau;
  double su = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double ui = (dir ? base[i] + s * dir[i] : base[i]) - tau;
    if (u) u[i] = ui;
    su += ui;
  }
  const double4 r0 = block_sum2_fin(su, 0.0, scr, [=](double x, double) { return make_double2((x - b) / (double)n, 0.0); });
  double theta = r0.z;
  double cnt = (double)n;
  for (int it = 0; it <= n; ++it) {
    double sa = 0.0;
    int ka = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double ui = u ? u[i] : (dir ? base[i] + s * dir[i] : base[i]) - tau;
      if (ui > theta) {
        sa += ui;
        ka += 1;
      }
    }
    const double4 r = block_sum2_fin(sa, (double)ka, scr, [=](double x, double y) {
      return make_double2(y > 0.0 ? (x - b) / y : 0.0, 0.0);
    });
    if (r.y == cnt || r.y == 0.0) break;
    cnt = r.y;
    theta = r.z;
  }
  return theta;
}

// (||x - Pi(x - g)||_2, that / max(norm, 1e-300)): the projected-simplex KKT
// residual and its relative value; tmp receives x - g - tau.
inline __device__ double2 kkt_residual_rel(const double* x, const double* g, int n, double tau, double* scr,
                                           double* tmp, double norm) {
  double s = 0.0;
  if (n > kSliceE * (int)blockDim.x) {
    const double th = slice_theta_mem(x, g, -1.0, n, tau, scr, tmp);  // tmp = (x - g) - tau
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double p = tau + fmax(tmp[i] - th, 0.0);
      const double e = x[i] - p;
      s += e * e;
    }
  } else {
    double uu[kSliceE];
    float uf[kSliceE];
    const double th = slice_theta_r(x, g, -1.0, n, tau, scr, tmp, uu, uf);
    const float thf = f32_trunc(th);
#pragma unroll
    for (int e = 0; e < kSliceE; ++e) {
      const int i = threadIdx.x + e * blockDim.x;
      if (i < n) {
        // p = tau + max(u - theta, 0): u - theta > 0 exactly when u > theta;
        // x - p is exactly 0 for x = p = tau
        const int c = gt_screen(uf[e], thf);
        const bool above = c > 0 || (c < 0 && uu[e] > th);
        const double xi = x[i];
        if (above || !same_bits(xi, tau)) {
          const double p = above ? tau + (uu[e] - th) : tau;
          const double d = xi - p;
          s += d * d;
        }
      }
    }
  }
  const double4 r = block_sum2_fin(s, 0.0, scr, [=](double x2, double) {
    const double k = sqrt(x2);
    return make_double2(k, k / fmax(norm, 1e-300));
  });
  return make_double2(r.z, r.w);
}

inline __device__ double kkt_residual(const double* x, const double* g, int n, double tau, double* scr, double* tmp) {
  return kkt_residual_rel(x, g, n, tau, scr, tmp, 1.0).x;
}

// ------------------------------------------------------- exact quartic step
__device__ __forceinline__ double dphi(const double* c, double a) {
  return ((4.0 * c[4] * a + 3.0 * c[3]) * a + 2.0 * c[2]) * a + c[1];
}
__device__ __forceinline__ double decrease(const double* c, double a) {
  return a * (c[1] + a * (c[2] + a * (c[3] + a * c[4])));
}

// The root of phi' in [lo, hi] (0 <= lo < hi) where phi' is monotone and
// changes sign (flo = phi'(lo) != 0), to adjacent doubles, by the 32 lanes of
// one warp (every lane calls; all return the same value).  Non-negative
// doubles are ordered like their bit patterns, so the bracket is searched in
// integer space: each round evaluates phi' at 31 points spaced evenly in the
// bit patterns strictly inside the bracket and keeps the sub-bracket where
// the sign changes (five bits per round, <= 13 rounds).  On this part a lone
// thread's dependent FP64 operation takes about as long as a whole warp's
// (the FP64 pipe is ~2 operations/clk/SM), so the 31 evaluations of a round
// cost about one bisection step.  Like bisection it ends at the midpoint of
// adjacent doubles bracketing the sign change (or at an exact zero of phi',
// the smallest one evaluated).
__device__ __forceinline__ double dphi_root_w(const double* c, double lo, double hi, double flo) {
  const int lane = threadIdx.x & 31;
  const bool neg = flo < 0.0;
  unsigned long long ia = (unsigned long long)__double_as_longlong(lo), ib = (unsigned long long)__double_as_longlong(hi);
  for (int it = 0; it < 16 && ib - ia > 1ull; ++it) {
    const unsigned long long span = ib - ia;
    // point j (j < 31): ia + floor(span (j + 1) / 32), without overflow
    auto point = [&](int j) -> unsigned long long {
      const unsigned long long q = (unsigned long long)(j + 1);
      return ia + (span >> 5) * q + (((span & 31ull) * q) >> 5);
    };
    const unsigned long long ij = point(lane);
    const bool valid = lane < 31 && ij > ia && ij < ib;
    const double x = __longlong_as_double((long long)ij);
    const double f = valid ? dphi(c, x) : 1.0;
    const unsigned zero = __ballot_sync(0xffffffffu, valid && f == 0.0);
    if (zero != 0u) return __shfl_sync(0xffffffffu, x, __ffs(zero) - 1);
    const unsigned los = __ballot_sync(0xffffffffu, valid && ((f < 0.0) == neg));
    const unsigned his = __ballot_sync(0xffffffffu, valid && !((f < 0.0) == neg));
    const int kh = his != 0u ? __ffs(his) - 1 : 31;  // first point on the side of hi
    const unsigned below = kh >= 31 ? los : (los & ((1u << kh) - 1u));
    const unsigned long long nb = kh < 31 ? point(kh) : ib;
    if (below != 0u) ia = point(31 - __clz(below));  // last point on the side of lo before it
    ib = nb;
  }
  const double a = __longlong_as_double((long long)ia), b = __longlong_as_double((long long)ib);
  return (a != b) ? 0.5 * (a + b) : a;
}

// Minimiser of A0 + A1 a + ... + A4 a^4 on [0, amax] (Prop. quartic exact line
// search): candidates 0, amax and the real roots of phi' in (0, amax).  The
// real roots of phi'' (cancellation-free quadratic formula) split the interval
// into pieces on which phi' is monotone; a sign change brackets one root,
// found to adjacent doubles (dphi_root_w).  Ties keep the smallest alpha.
// Warp-cooperative: every lane of one warp calls with the same arguments and
// receives the result.
inline __device__ double quartic_argmin_w(const double* c, double amax) {
  if (!(amax > 0.0)) return 0.0;
  double brk[4];
  int nb = 0;
  brk[nb++] = 0.0;
  {
    const double qa = 12.0 * c[4], qb = 6.0 * c[3], qc = 2.0 * c[2];
    double r1 = NAN, r2 = NAN;
    if (qa == 0.0) {
      if (qb != 0.0) r1 = -qc / qb;
    } else {
      const double disc = qb * qb - 4.0 * qa * qc;
      if (disc >= 0.0) {
        const double q = -0.5 * (qb + copysign(sqrt(disc), qb));
        r1 = q / qa;
        r2 = (q != 0.0) ? qc / q : 0.0;
      }
    }
    if (r1 > r2) {
      const double t = r1;
      r1 = r2;
      r2 = t;
    }
    if (r1 > 0.0 && r1 < amax) brk[nb++] = r1;
    if (r2 > 0.0 && r2 < amax && r2 != r1) brk[nb++] = r2;
  }
  brk[nb++] = amax;
  double cand[6];
  int nc = 0;
  cand[nc++] = 0.0;
  cand[nc++] = amax;
  for (int k = 0; k + 1 < nb; ++k) {
    const double lo = brk[k], hi = brk[k + 1];
    const double flo = dphi(c, lo), fhi = dphi(c, hi);
    if (flo == 0.0) { cand[nc++] = lo; continue; }
    if (fhi == 0.0) { cand[nc++] = hi; continue; }
    if ((flo < 0.0) == (fhi < 0.0)) continue;
    cand[nc++] = dphi_root_w(c, lo, hi, flo);
  }
  // sort ascending (tiny insertion sort), then keep the first strict minimum
  for (int i = 1; i < nc; ++i) {
    const double v = cand[i];
    int j = i - 1;
    while (j >= 0 && cand[j] > v) { cand[j + 1] = cand[j]; --j; }
    cand[j + 1] = v;
  }
  double best_a = 0.0, best_v = 0.0;
  for (int i = 0; i < nc; ++i) {
    const double a = cand[i];
    if (!(a >= 0.0 && a <= amax)) continue;
    if (i > 0 && a == cand[i - 1]) continue;
    const double v = decrease(c, a);
    if (v < best_v) { best_a = a; best_v = v; }
  }
  return best_a;
}

// Armijo backtracking on the same quartic (the paper's Armijo diagnostic,
// Table yand-line-search): the largest alpha = amax 2^-j, j < 60, with
// phi(alpha) - phi(0) <= 1e-4 alpha phi'(0); 0 when phi'(0) >= 0.  Lane j of
// the warp tests j and j + 32 (amax 2^-j formed by ldexp: the repeated
// halving, exactly, while it stays in the normal range).  Warp-cooperative.
inline __device__ double armijo_step_w(const double* c, double amax) {
  if (!(amax > 0.0) || !(c[1] < 0.0)) return 0.0;
  const int lane = threadIdx.x & 31;
  for (int j0 = 0; j0 < 60; j0 += 32) {
    const int j = j0 + lane;
    const double a = ldexp(amax, -j);
    const unsigned ok = __ballot_sync(0xffffffffu, j < 60 && decrease(c, a) <= 1e-4 * a * c[1]);
    if (ok != 0u) return ldexp(amax, -(j0 + __ffs(ok) - 1));
  }
  return 0.0;
}

// Step along a direction on [0, amax] by rule (SI_LSRULE); warp-cooperative.
inline __device__ double line_step_w(const double* c, double amax, int rule) {
  return rule == 1 ? armijo_step_w(c, amax) : quartic_argmin_w(c, amax);
}

// line_step_w by warp 0, broadcast through the shared *slot (the search is a
// chain of dependent FP64 operations, which every warp of the block would
// otherwise repeat on the FP64 pipe).  Block-uniform call.
inline __device__ double block_line_step(const double* c, double amax, int rule, double* slot) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const double v = line_step_w(c, amax, rule);
    if (threadIdx.x == 0) *slot = v;
  }
  __syncthreads();
  return *slot;
}

// ------------------------------------------------- SplitMix64 normal probes
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long index) {
  unsigned long long z = seed + (index + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Standard normal probe coordinate i of probe k at `iteration` (SplitMix64
// stream per probe; Box-Muller cosine branch on two 53-bit uniforms).
__device__ __forceinline__ double probe_value(unsigned long long seed, long long iteration, int k, int i) {
  const unsigned long long ps = splitmix64(seed, (unsigned long long)iteration * 256ull + (unsigned long long)k);
  const double u1 = ((double)(splitmix64(ps, 2ull * (unsigned long long)i) >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = ((double)(splitmix64(ps, 2ull * (unsigned long long)i + 1ull) >> 11) + 1.0) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// The same normal from the same two uniforms (their top 24 bits), by Box-Muller
// in FP32: the probes of FP32 Krylov recurrences.
__device__ __forceinline__ float probe_value_f(unsigned long long seed, long long iteration, int k, int i) {
  const unsigned long long ps = splitmix64(seed, (unsigned long long)iteration * 256ull + (unsigned long long)k);
  const float u1 = ((float)(splitmix64(ps, 2ull * (unsigned long long)i) >> 40) + 1.0f) * 0x1.0p-24f;
  const float u2 = ((float)(splitmix64(ps, 2ull * (unsigned long long)i + 1ull) >> 40) + 1.0f) * 0x1.0p-24f;
  return sqrtf(-2.0f * logf(u1)) * cosf(6.28318530717958648f * u2);
}

}  // namespace mvsk
