// Fused streaming passes over the centred return matrix A (T x ld, row-major).
//
// Every sample oracle of Prop. 1 (Eqs. operator-f/grad/hvp/third) and the
// power sums of Prop. (quartic exact line search) has the same shape: for
// each row a_t, take a few dot products a_t^T v_j, turn them (with the cached
// z_t) into row weights omega_t,m and scalar contributions, and accumulate
// sum_t omega_t,m a_t.  One pass reads each row of A from HBM exactly once:
//
//   * CTA b owns rows [b*rows_per_cta, (b+1)*rows_per_cta).  Chunks of RB rows
//     (RB * ld * sizeof(TA) = 8*ld bytes, contiguous) stream into a ring of
//     shared-memory stages with one cp.async.bulk per chunk, completing on an
//     mbarrier (bounded waits).
//   * Each thread owns the 16-byte column vectors tid, tid+512, ... of a row;
//     forward dot products are block-reduced (warp shuffles, then a fixed-order
//     sum over warps), the epilogue runs one thread per row, and the backward
//     accumulation of omega * a_t stays in registers.
//   * Each CTA writes its column partials; a second kernel sums them over CTAs
//     in a fixed order (deterministic results, no floating-point atomics).
//
// FP64 A keeps the input vectors in shared memory (the pass is bound by the
// FP64 pipe); FP32/BF16 A keep them in registers as FP32 and accumulate in
// FP32 (the pass is bound by HBM).
#pragma once

#include "common.cuh"

namespace mvsk {

enum PassMode : int {
  M_VALGRAD = 0,  // z_t = a_t.x (stored); omega = psi'(z); scalar: psi(z)
  M_FWD = 1,      // store a_t.v_j for each input (rowout[j*T + t])
  M_HVP = 2,      // omega_j = psi''(z_t) a_t.v_j
  M_HVPDIAG = 3,  // inputs (nu, 1_F): omega0 = psi'' a.nu ; out1 += psi'' a o a ; scalars psi''(a.nu)^2, psi''(a.1F)^2
  M_THIRD = 4,    // omega = psi'''(z) (a.u)(a.v)
  M_RHAT = 5,     // rowout[t] (+)= rscale * sum_q (a.v_2q)(a.v_2q+1)
  M_BACK = 6,     // omega = psi'''(z_t) roww[t]  (no forward products)
  M_LS = 7        // w = a.d ; twelve power sums s_rs of (z, w); rowout[t] = w if given
};

template <typename TA>
struct ATraits;
template <>
struct ATraits<double> {
  using acc = double;
  static constexpr int VEC = 2, RB = 1;
  static constexpr bool kInSmem = true;
};
template <>
struct ATraits<float> {
  using acc = float;
  static constexpr int VEC = 4, RB = 2;
  static constexpr bool kInSmem = false;
};
template <>
struct ATraits<__nv_bfloat16> {
  using acc = float;
  static constexpr int VEC = 8, RB = 4;
  static constexpr bool kInSmem = false;
};

constexpr int kMaxIn = 4;

struct PassArgs {
  const void* A;
  long long T;
  int ld;                      // elements per row (multiple of kPad)
  const double* in[kMaxIn];    // input vectors, ld values each, zero in padding
  const double* z;             // cached z (T), for modes that use it
  const double* roww;          // per-row weights (M_BACK)
  double* rowout;              // per-row outputs (see modes)
  int row_accum;               // M_RHAT: add to rowout instead of overwrite
  double c2, c3, c4;
  double rscale;
  void* part;                  // [gridDim.x][NOUT][ld] in ATraits::acc
  double* spart;               // [gridDim.x][NS]
  int rows_per_cta;
  int stages;
  int* err;
  const int* skip;             // when non-null and *skip != 0 the pass does nothing
  const int* live;             // when non-null and *live == 0 the pass does nothing
  int* counter;                // when non-null, incremented once by a pass that runs
};

template <typename TA>
__device__ __forceinline__ void load_avec(const TA* p, typename ATraits<TA>::acc (&a)[ATraits<TA>::VEC]);

template <>
__device__ __forceinline__ void load_avec<double>(const double* p, double (&a)[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a[0] = v.x;
  a[1] = v.y;
}
template <>
__device__ __forceinline__ void load_avec<float>(const float* p, float (&a)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a[0] = v.x;
  a[1] = v.y;
  a[2] = v.z;
  a[3] = v.w;
}
template <>
__device__ __forceinline__ void load_avec<__nv_bfloat16>(const __nv_bfloat16* p, float (&a)[8]) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 f = __bfloat1622float2(h[q]);
    a[2 * q] = f.x;
    a[2 * q + 1] = f.y;
  }
}

template <typename TA>
__host__ __device__ constexpr int kv_max() {
  return (kMaxCols / ATraits<TA>::VEC + kThreads - 1) / kThreads;
}

template <int MODE>
struct ModeShape;
template <> struct ModeShape<M_VALGRAD> { static constexpr int NOUT = 1, NS = 1; };
template <> struct ModeShape<M_FWD> { static constexpr int NOUT = 0, NS = 0; };
template <> struct ModeShape<M_HVP> { static constexpr int NOUT = -1, NS = 0; };   // NOUT = NIN
template <> struct ModeShape<M_HVPDIAG> { static constexpr int NOUT = 2, NS = 2; };
template <> struct ModeShape<M_THIRD> { static constexpr int NOUT = 1, NS = 0; };
template <> struct ModeShape<M_RHAT> { static constexpr int NOUT = 0, NS = 0; };
template <> struct ModeShape<M_BACK> { static constexpr int NOUT = 1, NS = 0; };
template <> struct ModeShape<M_LS> { static constexpr int NOUT = 0, NS = 12; };

template <int MODE, int NIN>
__host__ __device__ constexpr int mode_nout() {
  return ModeShape<MODE>::NOUT < 0 ? NIN : ModeShape<MODE>::NOUT;
}

// Shared-memory bytes of one pass launch with `stages` ring stages.
template <typename TA, int MODE, int NIN>
__host__ __device__ constexpr size_t pass_smem_fixed(int ld) {
  using acc = typename ATraits<TA>::acc;
  constexpr int RB = ATraits<TA>::RB;
  return (ATraits<TA>::kInSmem ? (size_t)NIN * ld * sizeof(double) : 0) +
         (size_t)kWarps * RB * (NIN > 0 ? NIN : 1) * sizeof(double) +
         (size_t)RB * (mode_nout<MODE, NIN>() + 1) * sizeof(acc) + 64 * sizeof(double) + 16 * sizeof(uint64_t) + 256;
}

template <typename TA, int MODE, int NIN>
__global__ void __launch_bounds__(kThreads, 1) rowpass_kernel(PassArgs p) {
  using acc = typename ATraits<TA>::acc;
  constexpr int VEC = ATraits<TA>::VEC;
  constexpr int RB = ATraits<TA>::RB;
  constexpr int KV = kv_max<TA>();
  constexpr int NOUT = mode_nout<MODE, NIN>();
  constexpr int NS = ModeShape<MODE>::NS;
  constexpr bool kInSmem = ATraits<TA>::kInSmem;
  constexpr int NINR = NIN > 0 ? NIN : 1;
  constexpr int NOUTR = NOUT > 0 ? NOUT : 1;
  constexpr int NSR = NS > 0 ? NS : 1;

  if (p.skip != nullptr && *p.skip != 0) return;
  if (p.live != nullptr && *p.live == 0) return;
  if (p.counter != nullptr && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(p.counter, 1);

  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ld = p.ld;
  const int NV = ld / VEC;
  const size_t stage_bytes = (size_t)RB * ld * sizeof(TA);
  unsigned char* stages = smem_raw;
  unsigned char* cur = smem_raw + stage_bytes * p.stages;
  double* sin = reinterpret_cast<double*>(cur);  // FP64: NIN input vectors
  if (kInSmem) cur += (size_t)NIN * ld * sizeof(double);
  double* red = reinterpret_cast<double*>(cur);
  cur += (size_t)kWarps * RB * NINR * sizeof(double);
  acc* wts = reinterpret_cast<acc*>(cur);
  cur += (size_t)RB * (NOUT + 1) * sizeof(acc);
  cur = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(cur) + 15) & ~uintptr_t(15));
  double* scr = reinterpret_cast<double*>(cur);
  cur += 64 * sizeof(double);
  uint64_t* bar = reinterpret_cast<uint64_t*>(cur);
  __shared__ int s_abort;
  __shared__ int s_issued;

  const long long r0 = (long long)blockIdx.x * p.rows_per_cta;
  const long long r1 = r0 + p.rows_per_cta < p.T ? r0 + p.rows_per_cta : p.T;
  const int nrows = r1 > r0 ? (int)(r1 - r0) : 0;
  const int nchunks = (nrows + RB - 1) / RB;
  const TA* Ab = reinterpret_cast<const TA*>(p.A) + (size_t)r0 * ld;

  if (tid == 0) {
    s_abort = 0;
    s_issued = 0;
    for (int s = 0; s < p.stages; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
  }
  // Input vectors.
  acc xin[kInSmem ? 1 : NINR][kInSmem ? 1 : KV][VEC];
  if constexpr (kInSmem) {
    for (int j = 0; j < NIN; ++j)
      for (int i = tid; i < ld; i += kThreads) sin[j * ld + i] = p.in[j][i];
  } else {
#pragma unroll
    for (int j = 0; j < NINR; ++j)
#pragma unroll
      for (int k = 0; k < KV; ++k) {
        const int v = tid + k * kThreads;
#pragma unroll
        for (int e = 0; e < VEC; ++e)
          xin[j][k][e] = (j < NIN && v < NV) ? (acc)p.in[j][v * VEC + e] : (acc)0;
      }
  }
  acc yout[NOUTR][KV][VEC];
#pragma unroll
  for (int m = 0; m < NOUTR; ++m)
#pragma unroll
    for (int k = 0; k < KV; ++k)
#pragma unroll
      for (int e = 0; e < VEC; ++e) yout[m][k][e] = (acc)0;
  double sacc[NSR];
#pragma unroll
  for (int s = 0; s < NSR; ++s) sacc[s] = 0.0;
  __syncthreads();

  auto issue = [&](int c) {
    const int s = c % p.stages;
    const int rows = nrows - c * RB < RB ? nrows - c * RB : RB;
    const uint32_t bytes = (uint32_t)((size_t)rows * ld * sizeof(TA));
    mbar_expect_tx(&bar[s], bytes);
    bulk_g2s(stages + (size_t)s * stage_bytes, Ab + (size_t)c * RB * ld, bytes, &bar[s]);
  };
  if (tid == 0) {
    const int pro = nchunks < p.stages ? nchunks : p.stages;
    for (int c = 0; c < pro; ++c) issue(c);
    s_issued = pro;
  }

  int consumed = -1;
  for (int c = 0; c < nchunks; ++c) {
    const int s = c % p.stages;
    const uint32_t parity = (uint32_t)((c / p.stages) & 1);
    if (!mbar_wait_bounded(&bar[s], parity)) s_abort = 1;
    const int rows = nrows - c * RB < RB ? nrows - c * RB : RB;
    const TA* buf = reinterpret_cast<const TA*>(stages + (size_t)s * stage_bytes);

    if constexpr (NIN > 0) {
      acc pd[RB][NINR];
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int j = 0; j < NINR; ++j) pd[r][j] = (acc)0;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        if (r < rows) {
#pragma unroll
          for (int k = 0; k < KV; ++k) {
            const int v = tid + k * kThreads;
            if (v < NV) {
              acc a[VEC];
              load_avec<TA>(buf + (size_t)r * ld + v * VEC, a);
#pragma unroll
              for (int j = 0; j < NIN; ++j) {
                if constexpr (kInSmem) {
                  const double2 xv = *reinterpret_cast<const double2*>(sin + j * ld + v * VEC);
                  pd[r][j] = fma(a[0], xv.x, pd[r][j]);
                  pd[r][j] = fma(a[1], xv.y, pd[r][j]);
                } else {
#pragma unroll
                  for (int e = 0; e < VEC; ++e) pd[r][j] = fma(a[e], xin[j][k][e], pd[r][j]);
                }
              }
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int j = 0; j < NIN; ++j) {
          const acc t = warp_sum(pd[r][j]);
          if (lane == 0) red[(warp * RB + r) * NINR + j] = (double)t;
        }
    }
    __syncthreads();  // (1) dots in red; every thread finished chunk c-1
    if (s_abort) break;
    consumed = c;
    if (tid == 0 && c >= 1) {
      const int nc = c - 1 + p.stages;
      if (nc < nchunks) {
        issue(nc);
        s_issued = nc + 1;
      }
    }
    if (tid < rows) {
      const long long t = r0 + (long long)c * RB + tid;
      double dot[NINR];
#pragma unroll
      for (int j = 0; j < NINR; ++j) {
        double s2 = 0.0;
        if (j < NIN)
          for (int w = 0; w < kWarps; ++w) s2 += red[(w * RB + tid) * NINR + j];
        dot[j] = s2;
      }
      const Psi psi{p.c2, p.c3, p.c4};
      double om[NOUTR];
#pragma unroll
      for (int m = 0; m < NOUTR; ++m) om[m] = 0.0;
      if constexpr (MODE == M_VALGRAD) {
        const double zt = dot[0];
        p.rowout[t] = zt;
        om[0] = psi.d1(zt);
        sacc[0] += psi.f(zt);
      } else if constexpr (MODE == M_FWD) {
#pragma unroll
        for (int j = 0; j < NIN; ++j) p.rowout[(size_t)j * p.T + t] = dot[j];
      } else if constexpr (MODE == M_HVP) {
        const double h = psi.d2(p.z[t]);
#pragma unroll
        for (int j = 0; j < NIN; ++j) om[j] = h * dot[j];
      } else if constexpr (MODE == M_HVPDIAG) {
        const double h = psi.d2(p.z[t]);
        om[0] = h * dot[0];
        om[1] = h;
        sacc[0] += h * dot[0] * dot[0];
        sacc[1] += h * dot[1] * dot[1];
      } else if constexpr (MODE == M_THIRD) {
        om[0] = psi.d3(p.z[t]) * dot[0] * dot[1];
      } else if constexpr (MODE == M_RHAT) {
        double s2 = 0.0;
#pragma unroll
        for (int q = 0; q < NIN / 2; ++q) s2 += dot[2 * q] * dot[2 * q + 1];
        s2 *= p.rscale;
        p.rowout[t] = p.row_accum ? p.rowout[t] + s2 : s2;
      } else if constexpr (MODE == M_BACK) {
        om[0] = psi.d3(p.z[t]) * p.roww[t];
      } else if constexpr (MODE == M_LS) {
        const double zt = p.z[t], w = dot[0];
        if (p.rowout != nullptr) p.rowout[t] = w;
        const double z2 = zt * zt, w2 = w * w;
        sacc[0] += z2;           // s20
        sacc[1] += z2 * zt;      // s30
        sacc[2] += z2 * z2;      // s40
        sacc[3] += zt * w;       // s11
        sacc[4] += z2 * w;       // s21
        sacc[5] += z2 * zt * w;  // s31
        sacc[6] += w2;           // s02
        sacc[7] += zt * w2;      // s12
        sacc[8] += z2 * w2;      // s22
        sacc[9] += w2 * w;       // s03
        sacc[10] += zt * w2 * w; // s13
        sacc[11] += w2 * w2;     // s04
      }
#pragma unroll
      for (int m = 0; m < NOUT; ++m) wts[tid * (NOUT + 1) + m] = (acc)om[m];
    }
    __syncthreads();  // (2) weights visible
    if constexpr (NOUT > 0) {
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        if (r < rows) {
          acc w[NOUTR];
#pragma unroll
          for (int m = 0; m < NOUT; ++m) w[m] = wts[r * (NOUT + 1) + m];
#pragma unroll
          for (int k = 0; k < KV; ++k) {
            const int v = tid + k * kThreads;
            if (v < NV) {
              acc a[VEC];
              load_avec<TA>(buf + (size_t)r * ld + v * VEC, a);
              if constexpr (MODE == M_HVPDIAG) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                  yout[0][k][e] = fma(w[0], a[e], yout[0][k][e]);
                  yout[1][k][e] = fma(w[1] * a[e], a[e], yout[1][k][e]);
                }
              } else {
#pragma unroll
                for (int m = 0; m < NOUT; ++m)
#pragma unroll
                  for (int e = 0; e < VEC; ++e) yout[m][k][e] = fma(w[m], a[e], yout[m][k][e]);
              }
            }
          }
        }
      }
    }
  }

  if (s_abort) {
    // Drain: wait (bounded) for every copy still in flight, then leave.
    if (tid == 0) {
      atomicOr(p.err, kErrWaitTimeout);
      for (int c = consumed + 1; c < s_issued; ++c) {
        if (!mbar_wait_bounded(&bar[c % p.stages], (uint32_t)((c / p.stages) & 1))) {
          atomicOr(p.err, kErrDrainTimeout);
          break;
        }
      }
    }
    __syncthreads();
    return;
  }

  if constexpr (NOUT > 0) {
    acc* part = reinterpret_cast<acc*>(p.part) + (size_t)blockIdx.x * NOUT * ld;
#pragma unroll
    for (int m = 0; m < NOUT; ++m)
#pragma unroll
      for (int k = 0; k < KV; ++k) {
        const int v = tid + k * kThreads;
        if (v < NV) {
#pragma unroll
          for (int e = 0; e < VEC; ++e) part[(size_t)m * ld + v * VEC + e] = yout[m][k][e];
        }
      }
  }
  if constexpr (NS > 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double t = block_sum(sacc[s], scr);
      if (tid == 0) p.spart[(size_t)blockIdx.x * NS + s] = t;
    }
  }
}

}  // namespace mvsk
