// C ABI of libmvsk (see include/mvsk.h): context, centring, the YAND-MVSK
// driver (Alg. 1) and the oracle exports.  Host code orchestrates; every
// arithmetic step of the method runs in the kernels of this library.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "dense.cuh"
#include "gemm_tc.cuh"
#include "internal.h"
#include "ozaki.cuh"
#include "mvsk.h"
#include "solver_kernels.cuh"

using namespace mvsk;

namespace {

thread_local char g_err[512];

struct Options {
  double tau = 1e-8, eta = 0.05, max_elapsed = 60.0, krylov_tol = 1e-3, reg = NAN;
  double restart_eta1 = 0.045, restart_eta2 = 0.02, release_ratio = 0.5, eps_act = 1e-15;
  double descent_eps = 1e-10, stall_factor = 0.99, cal_rel_tol = 1e-9, cal_bracket_tol = 1e-12;
  int max_iter = 300, pcg_max_iter = 40, restart_iter1 = 120, restart_iter2 = 120, krylov_maxit = 15, probes = 8;
  int stall_window = 10, pref_scaling = 1, oracle_prec = 0, arc_halvings = 40, cal_max_evals = 40, trace = 0;
  int split_products = 1;  // batched solves: FP64 products on the tensor cores (ozaki.cuh)
  int batch_lanes = 0;     // batched solves: concurrent instances (0: all requests at once)
  int line_search = 0;     // 0 exact quartic step, 1 Armijo backtracking on the quartic
  int group_cal = 1;       // batched solves: requests sharing (c2, c3, c4) start calibration on a c1 grid
  int face_products = 1;   // batched solves: direction products restricted to the union of the faces
  int face_small = 1;      // ... and, when every face is small, explicit face Grams instead of the products
  unsigned long long probe_seed = 0x5EEDull;
};

// Instance-strided state of a lockstep batch (see batch_impl.cuh).
struct BatchBuf {
  int cap = 0;
  mvsk::Inst base{};
  std::vector<void*> mem;
  // pinned host copies of the lanes' state words and evaluations (read every
  // iteration: asynchronous copies, one synchronisation)
  int* si_h = nullptr;
  double* sd_h = nullptr;
  int* q_si = nullptr;      // per request: the state words at its end
  double* q_ev = nullptr;   // per request: f, KKT residual, mu^T x, kkt0
  int qhcap = 0;
  // switch handle of the one-graph iteration (valid while has_cond is set during its capture)
  cudaGraphConditionalHandle cond = 0;
  int has_cond = 0;
  double* ev_h = nullptr;
  int hcap = 0;
  __nv_bfloat16* P16 = nullptr;
  __nv_bfloat16* S16T = nullptr;
  float* part = nullptr;
  size_t part_floats = 0;
  double* Wt = nullptr;  // psi'(z) of every instance (T-strided), right-hand side of A^T W
  double* G0 = nullptr;  // T^-1 A^T psi'_b(A 1/n) of every instance (ld-strided): gradient at 1/n less c1 mu
  __nv_bfloat16* H16 = nullptr;  // psi''_b(z_b) of every instance (Tp-strided BF16)
  float* Hf = nullptr;           // the same in FP32 (T-strided)
  std::vector<int> kq_idx;       // inner solves started since the last KKT0 flush
  std::vector<double> kq_c1;
  void* kq_dev = nullptr;        // device copy: c1 (cap doubles) then indices
  int* need = nullptr;   // any instance needs the second line-search product
  double* Gq = nullptr;  // G0 of every request when requests queue for fewer lanes (qcap x ld)
  double* wls = nullptr;    // projected line-search direction A d of every instance (T-strided)
  double* zsave = nullptr;  // cached z of the warm-start brackets lo, hi (2 x T per instance)
  double* z0 = nullptr;     // A 1/n (T)
  int* needz = nullptr;     // the next iteration recomputes z = A x (device flag)
  int needz_req = 0;        // host: a start without a cached z asks for that
  double* Wq = nullptr;     // user warm starts of the requests (wcap x ld) ...
  double* Zq = nullptr;     // ... and their A w0 (wcap x T)
  int wcap = 0;
  double* gpool = nullptr;  // calibration grid points: x* (ld) and z (T) per lane
  int gcap = 0;
  // face-restricted direction products (batch_impl.cuh): the gathered columns
  // of A in the union U of the faces (T x ld and ld x Tp BF16, A^2 rows),
  // flags, U itself, positions in U, {|U|, padded |U|}, runtime extents of
  // the product specs (device) and the specs themselves (host copy)
  __nv_bfloat16 *u_AU = nullptr, *u_AUT = nullptr, *u_A2UT = nullptr;
  int *u_flag = nullptr, *u_idx = nullptr, *u_pos = nullptr, *u_info = nullptr, *u_rt = nullptr;
  __nv_bfloat16* u_AFU = nullptr;  // digit planes of A's columns in U (split line-search product)
  mvsk::UProd* u_specs = nullptr;
  std::vector<mvsk::UProd> u_hspec;
  bool umode = false;
  // small-face direction block (face_small.cuh): face lists (ld ints per
  // instance), partial and final face Grams, partial Hutchinson corrections
  int* f_list = nullptr;
  float *f_gp = nullptr, *f_gram = nullptr, *f_ap = nullptr;
  int qcap = 0;
};

// Digit planes and buffers of the emulated-FP64 tensor-core products (ozaki.cuh).
struct OzBuf {
  __nv_bfloat16* AF = nullptr;  // digits of the rows of A: kOzS planes of MpF x ld
  __nv_bfloat16* AB = nullptr;  // digits of the columns of A: kOzS planes of MpB x ldT
  int* eF = nullptr;            // row exponents (MpF)
  int* eB = nullptr;            // column exponents (MpB)
  __nv_bfloat16* XF = nullptr;  // right-hand digits, kOzS*kOzMaxB rows x ld
  __nv_bfloat16* XB = nullptr;  // right-hand digits, kOzS*kOzMaxB rows x ldT
  int* fF = nullptr;            // right-hand exponents (kOzMaxB)
  int* fB = nullptr;
  long long* part = nullptr;    // split partials
  long long MpF = 0, ldT = 0;
  int MpB = 0, bp = 0;          // bp: vector count the right-hand maps are encoded for
  CUtensorMap tmXF, tmXB;
};

}  // namespace

struct mvsk_ctx {
  long long T = 0;
  int n = 0, ld = 0;
  uint32_t flags = 0;
  int dir_prec = P64;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;  // blocking stream created by the context (capturable)
  bool use_graphs = true;
  int nsm = 0, grid = 0, rows_per_cta = 0;
  double* A64 = nullptr;
  void* Alo = nullptr;  // BF16 or FP32 copy
  double* mu = nullptr;
  // per-instance device state (single instance)
  Inst in{};
  double* sd = nullptr;
  int* si = nullptr;
  void* part = nullptr;     // column partials (FP64-sized)
  double* spart = nullptr;  // scalar partials
  double* fwd = nullptr;    // per-row scratch [4][T]
  double* hd = nullptr;     // Gnu | diagG
  double* vec_scratch = nullptr;  // host<->device staging for vector arguments
  int* err = nullptr;
  int* hword = nullptr;     // pinned host words: [0] the error word's copy, [1] the direction form
  int ncolmax = 0;
  // preferences
  bool prefs_set = false;
  double lam[4] = {0, 0, 0, 0};
  double target = NAN;
  double c[4] = {0, 0, 0, 0};
  double s_equal = NAN;  // sqrt(m2(1/n))
  double mu_absmax = 0.0;
  Options opt;
  std::vector<void*> allocs;
  // profiling of the streaming passes
  bool prof_on = false;
  long long launches = 0;
  // dense buffers of the direct configuration (allocated at its first use)
  double *Gm = nullptr, *Bm = nullptr, *Ub = nullptr, *Rb = nullptr, *Pb = nullptr, *GC = nullptr, *Yb = nullptr;
  double* dvec = nullptr;
  int* dflag = nullptr;
  // K-major BF16 operands of the tensor-core products (n x Tp, Tp = T rounded up to 8)
  __nv_bfloat16* A16T = nullptr;
  __nv_bfloat16* W16T = nullptr;
  __nv_bfloat16* A2_16T = nullptr;  // bf16(a_ti^2), n x Tp (diagonal of the weighted Gram)
  long long Tp = 0;
  // tensor-core PCG products: BF16 columns, S^T, split-K partials, cached tensor maps
  __nv_bfloat16* P16 = nullptr;
  __nv_bfloat16* S16T = nullptr;
  float* part32 = nullptr;
  CUtensorMap tm_A16, tm_P16, tm_A16T, tm_S16T;
  BatchBuf batch;
  OzBuf oz;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;  // kind id per event pair
  size_t ev_used = 0;
  size_t ev_graph_begin = 0, ev_graph_end = 0;  // pairs captured into the current graph
  std::vector<char> ev_in_graph;                 // pair recorded as a graph node (folded per replay)
  std::vector<long long> prof_n;                 // accumulated launches per kind id
  std::vector<double> prof_ms;                   // accumulated device ms per kind id
  std::vector<double> prof_work;                 // accumulated algorithmic bytes (passes) or flops (GEMMs)
  std::vector<double> ev_work;                   // work of each recorded pair
  std::vector<char> ev_uscale;                   // work given per unit of |U| (face-restricted products)
  const int* prof_uinfo = nullptr;               // device {|U|, padded |U|} of the current batch
  std::vector<char> prof_sel;                    // kinds recorded (mvsk_profile_only); empty = all
  bool prof_open = false;                        // a begun pair awaits its end event
  int prof_stride = 1;                           // bracket every k-th selected launch (mvsk_profile_stride)
  std::vector<long long> prof_count;             // selected launches of each kind seen since enabling
};

namespace {

mvsk_status fail(mvsk_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

#define CU(call)                                                                                \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return fail(MVSK_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define TRY(expr)                  \
  do {                             \
    mvsk_status s_ = (expr);       \
    if (s_ != MVSK_OK) return s_;  \
  } while (0)

mvsk_status dalloc(mvsk_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MVSK_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  e = cudaMemsetAsync(*p, 0, bytes < 16 ? 16 : bytes, c->stream);
  if (e != cudaSuccess) return fail(MVSK_ECUDA, "cudaMemset: %s", cudaGetErrorString(e));
  return MVSK_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy n doubles from a caller pointer (host or device) into device dst (ld padded with zeros).
mvsk_status upload_vec(mvsk_ctx* c, double* dst, const double* src, int n) {
  CU(cudaMemsetAsync(dst, 0, sizeof(double) * c->ld, c->stream));
  CU(cudaMemcpyAsync(dst, src, sizeof(double) * n, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c->stream));
  return MVSK_OK;
}

mvsk_status download_vec(mvsk_ctx* c, double* dst, const double* src, size_t n) {
  CU(cudaMemcpyAsync(dst, src, sizeof(double) * n, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->stream));
  return MVSK_OK;
}

// Waits for the stream; the error word comes back by an asynchronous copy
// into pinned memory queued ahead of the wait (one round trip).
mvsk_status sync(mvsk_ctx* c) {
  CU(cudaMemcpyAsync(c->hword, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  const int e = c->hword[0];
  if (e != 0) {
    c->hword[0] = 0;
    cudaMemset(c->err, 0, sizeof(int));
    return fail(MVSK_ECUDA, "in-kernel bounded wait ran out (error word %d)", e);
  }
  return MVSK_OK;
}

// ----------------------------------------------------------------- kernels
__global__ void k_colmean(const double* R, long long T, int n, int ld, double* mu) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  // fixed-order two-level sum: chunks of 256 rows, then the chunk sums
  double tot = 0.0;
  for (long long t0 = 0; t0 < T; t0 += 256) {
    double s = 0.0;
    const long long t1 = t0 + 256 < T ? t0 + 256 : T;
    for (long long t = t0; t < t1; ++t) s += R[(size_t)t * ld + j];
    tot += s;
  }
  mu[j] = tot / (double)T;
}

// sigma[j] = sqrt(T^-1 sum_t A[t][j]^2) of the centred panel (population
// standard deviation of column j), in the order of k_colmean.
__global__ void k_colstd(const double* A, long long T, int n, int ld, double* sigma) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double tot = 0.0;
  for (long long t0 = 0; t0 < T; t0 += 256) {
    double s = 0.0;
    const long long t1 = t0 + 256 < T ? t0 + 256 : T;
    for (long long t = t0; t < t1; ++t) {
      const double a = A[(size_t)t * ld + j];
      s += a * a;
    }
    tot += s;
  }
  sigma[j] = sqrt(tot / (double)T);
}

template <typename TL>
__global__ void k_centre(double* A, TL* lo, long long T, int n, int ld, const double* mu, int* bad) {
  const size_t total = (size_t)T * ld;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q % ld);
    double v = 0.0;
    if (j < n) {
      v = A[q];
      if (!isfinite(v)) *bad = 1;
      v -= mu[j];
    }
    A[q] = v;
    if (lo != nullptr) lo[q] = (TL)v;
  }
}
template <>
__global__ void k_centre<__nv_bfloat16>(double* A, __nv_bfloat16* lo, long long T, int n, int ld, const double* mu,
                                        int* bad) {
  const size_t total = (size_t)T * ld;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q % ld);
    double v = 0.0;
    if (j < n) {
      v = A[q];
      if (!isfinite(v)) *bad = 1;
      v -= mu[j];
    }
    A[q] = v;
    lo[q] = __double2bfloat16(v);
  }
}

__global__ void __launch_bounds__(kVT) k_sumsq(const double* z, long long T, double* out) {
  __shared__ double scr[80];
  double s = 0.0;
  for (long long t = threadIdx.x; t < T; t += blockDim.x) s += z[t] * z[t];
  s = block_sum2(s, 0.0, scr).x;
  if (threadIdx.x == 0) *out = s;
}

__global__ void __launch_bounds__(kVT) k_project(const double* v, int n, double tau, double* out) {
  __shared__ double scr[80];
  const double th = slice_theta(v, nullptr, 0.0, n, tau, scr);
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = tau + fmax(v[i] - tau - th, 0.0);
}

__global__ void k_quartic(const double* coef, double amax, double* out) {
  const double v = quartic_argmin_w(coef, amax);  // one warp
  if (threadIdx.x == 0) *out = v;
}

__global__ void __launch_bounds__(kVT) k_alpha_max(const double* x, const double* d, int n, double tau, double* out) {
  __shared__ double scr[80];
  double am = INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (d[i] < 0.0) am = fmin(am, (x[i] - tau) / (-d[i]));
  am = block_min(am, scr);
  if (threadIdx.x == 0) *out = am;
}

__global__ void __launch_bounds__(kVT) k_ls_coef_only(Inst s, const double* spart, int G, const double* dir, double* out) {
  __shared__ double scr[80];
  __shared__ double ps[16];
  __shared__ double coef[5];
  // A0 from the power sums themselves (proof of Prop. quartic): -c1 mu^T x + c2 s20 - c3 s30 + c4 s40
  reduce_spart(spart, G, 12, s.sd[SD_INVT], ps);
  double mx = 0.0, md = 0.0;
  for (int i = threadIdx.x; i < s.n; i += blockDim.x) {
    mx += s.mu[i] * s.x[i];
    md += s.mu[i] * dir[i];
  }
  const double2 r = block_sum2(mx, md, scr);
  if (threadIdx.x == 0) {
    const double c1 = s.sd[SD_C1], c2 = s.sd[SD_C2], c3 = s.sd[SD_C3], c4 = s.sd[SD_C4];
    out[0] = -c1 * r.x + c2 * ps[0] - c3 * ps[1] + c4 * ps[2];
    out[1] = -c1 * r.y + 2.0 * c2 * ps[3] - 3.0 * c3 * ps[4] + 4.0 * c4 * ps[5];
    out[2] = c2 * ps[6] - 3.0 * c3 * ps[7] + 6.0 * c4 * ps[8];
    out[3] = -c3 * ps[9] + 4.0 * c4 * ps[10];
    out[4] = c4 * ps[11];
  }
  (void)coef;
}

__global__ void k_init_state(Inst s0, double tol, double eta, int maxit, int pcg, int stallwin, int probes,
                             unsigned long long seed, int kmaxit, int arcmax, int lsrule, const double* opts9) {
  Inst s = inst_at(s0, blockIdx.y);
  if (threadIdx.x != 0) return;
  for (int q = 0; q < kSI; ++q) s.si[q] = 0;
  for (int q = SD_HIST; q < kSD; ++q) s.sd[q] = 0.0;
  s.sd[SD_TOL] = tol;
  s.sd[SD_ETA] = eta;
  s.sd[SD_BEST] = INFINITY;
  s.sd[SD_TAU] = opts9[0];
  s.sd[SD_EPSACT] = opts9[1];
  s.sd[SD_RELRATIO] = opts9[2];
  s.sd[SD_REG] = opts9[3];
  s.sd[SD_KTOL] = opts9[4];
  s.sd[SD_C1] = opts9[5];
  s.sd[SD_C2] = opts9[6];
  s.sd[SD_C3] = opts9[7];
  s.sd[SD_C4] = opts9[8];
  s.sd[SD_INVT] = opts9[9];
  s.sd[SD_DESCEPS] = opts9[10];
  s.sd[SD_STALLF] = opts9[11];
  s.si[SI_MAXIT] = maxit;
  s.si[SI_PCG] = pcg;
  s.si[SI_STALLWIN] = stallwin;
  s.si[SI_PROBES] = probes;
  s.si[SI_SEEDLO] = (int)(unsigned)(seed & 0xffffffffull);
  s.si[SI_SEEDHI] = (int)(unsigned)(seed >> 32);
  s.si[SI_KMAXIT] = kmaxit;
  s.si[SI_ARCMAX] = arcmax;
  s.si[SI_LSRULE] = lsrule;
}

// A new phase of the PCG configuration: projected step eta, maxit iterations,
// and the stall window (0: no stall test, the last phase, which has no
// restart after it and runs until the tolerance or its iteration budget).
__global__ void k_new_phase(Inst s0, double eta, int maxit, int stallwin) {
  Inst s = inst_at(s0, blockIdx.y);
  if (threadIdx.x != 0) return;
  s.si[SI_DONE] = 0;
  s.si[SI_PHASEIT] = 0;
  s.si[SI_HISTN] = 0;
  s.si[SI_MAXIT] = maxit;
  s.si[SI_STALLWIN] = stallwin;
  s.sd[SD_ETA] = eta;
}

// ---------------------------------------------------------------- passes
PassArgs pass_args(mvsk_ctx* c) {
  PassArgs a;
  memset(&a, 0, sizeof(a));
  a.c2 = c->c[1];
  a.c3 = c->c[2];
  a.c4 = c->c[3];
  a.rscale = 1.0;
  return a;
}

// Profiling: kind ids 0..383 are streaming passes ((prec*16 + mode)*8 + nin);
// 400 + bn are tensor-core products with N tile bn; 680..685 the split FP64
// products (A V, A^T V, the same gated by a device flag, A V on the union of
// the faces, the same gated); 700 + i the named kernels of kKernelNames.
constexpr int kProfKinds = 760;
constexpr int kKindNamed = 700;
const char* const kKernelNames[] = {"k_face", "k_probe_fill", "k_pcg_setup", "k_pcg_step", "k_cols_bf16_b",
                                    "k_reduce_hvp1_b", "k_reduce_hvp2_b", "k_reduce_rhat_b", "k_pcg_setup2",
                                    "k_assemble", "k_decide1", "k_decide2", "k_end_iter", "k_oz_fin_z",
                                    "k_oz_fin_g", "k_oz_fin_ls", "k_oz_split_vecs", "k_need_ls2", "k_reduce_cols",
                                    "k_hd_cols", "k_hd_reduce1", "k_hd_reduce2", "k_hd_reduce_diag",
                                    "k_pcg_step_a", "k_z_step", "k_union", "k_gather_u", "k_face_list",
                                    "k_face_gram", "k_pcg_round", "k_face_hutch", "k_oz_split_u", "k_face_gram_fin",
                                    "k_pcg_setup_cols"};
enum NamedKernel : int {
  NK_FACE, NK_PROBE_FILL, NK_PCG_SETUP, NK_PCG_STEP, NK_COLS, NK_HVP1, NK_HVP2, NK_RHAT, NK_PCG_SETUP2, NK_ASSEMBLE,
  NK_DECIDE1, NK_DECIDE2, NK_END_ITER, NK_OZ_Z, NK_OZ_G, NK_OZ_LS, NK_OZ_SPLIT, NK_NEED, NK_REDUCE_COLS, NK_HD_COLS,
  NK_HD_RED1, NK_HD_RED2, NK_HD_DIAG, NK_PCG_STEP_A, NK_ZSTEP, NK_UNION, NK_GATHER, NK_FACE_LIST, NK_GRAM, NK_PCG_ROUND,
  NK_HUTCH, NK_OZ_SPLIT_U, NK_GRAM_FIN, NK_PCG_SETUP_COLS, NK_COUNT
};
static_assert(sizeof(kKernelNames) / sizeof(kKernelNames[0]) == NK_COUNT && kKindNamed + NK_COUNT <= kProfKinds,
              "named kernel kinds");

mvsk_status prof_begin(mvsk_ctx* c, int kind, double work) {
  if (!c->prof_on || (!c->prof_sel.empty() && !c->prof_sel[kind])) return MVSK_OK;
  if (c->prof_count.empty()) c->prof_count.assign(kProfKinds, 0);
  if (c->prof_count[kind]++ % c->prof_stride != 0) return MVSK_OK;
  c->prof_open = true;
  if (c->prof_n.empty()) {
    c->prof_n.assign(kProfKinds, 0);
    c->prof_ms.assign(kProfKinds, 0.0);
    c->prof_work.assign(kProfKinds, 0.0);
  }
  c->ev_work.push_back(work);
  c->ev_uscale.push_back(0);
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  CU(cudaStreamIsCapturing(c->stream, &cst));
  c->ev_in_graph.push_back(cst == cudaStreamCaptureStatusActive ? 1 : 0);
  if (c->ev_used + 2 > c->ev_pool.size()) {
    for (int q = 0; q < 512; ++q) {
      cudaEvent_t e;
      CU(cudaEventCreate(&e));
      c->ev_pool.push_back(e);
    }
  }
  c->ev_kind.push_back(kind);
  // Inside a capture a plain record only orders streams; External makes it a graph node.
  CU(cudaEventRecordWithFlags(c->ev_pool[c->ev_used], c->stream,
                              c->ev_in_graph.back() ? cudaEventRecordExternal : cudaEventRecordDefault));
  return MVSK_OK;
}

mvsk_status prof_end(mvsk_ctx* c) {
  if (!c->prof_on || !c->prof_open) return MVSK_OK;
  c->prof_open = false;
  CU(cudaEventRecordWithFlags(c->ev_pool[c->ev_used + 1], c->stream,
                              c->ev_in_graph.back() ? cudaEventRecordExternal : cudaEventRecordDefault));
  c->ev_used += 2;
  return MVSK_OK;
}

// Launch statement `launch` bracketed by profiler events of named kernel nk.
#define PROF_LAUNCH(nk, launch)                    \
  do {                                             \
    TRY(prof_begin(c, kKindNamed + (nk), 0.0));    \
    launch;                                        \
    CU(cudaGetLastError());                        \
    TRY(prof_end(c));                              \
    c->launches += 1;                              \
  } while (0)

// A pair whose work is given per unit of the padded |U| of the iteration
// (face-restricted products: their K or their output rows is |U|).
mvsk_status prof_begin_u(mvsk_ctx* c, int kind, double work_per_unit) {
  const size_t before = c->ev_kind.size();
  TRY(prof_begin(c, kind, work_per_unit));
  if (c->ev_kind.size() > before) c->ev_uscale.back() = 1;
  return MVSK_OK;
}

// Fold the event pairs [b, e) into the per-kind totals (stream must be idle).
// Event pairs [b, e) after the stream has passed them; union-scaled work is
// multiplied by the union size, read from uinfo_host when given (a copy
// queued before the wait), else from the device.
mvsk_status prof_collect(mvsk_ctx* c, size_t b, size_t e, const int* uinfo_host = nullptr) {
  double units = uinfo_host != nullptr ? (double)uinfo_host[1] : -1.0;
  for (size_t q = b; q < e; ++q) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, c->ev_pool[2 * q], c->ev_pool[2 * q + 1]));
    double w = c->ev_work[q];
    if (c->ev_uscale[q]) {
      if (units < 0.0) {
        int info[2] = {0, 0};
        if (c->prof_uinfo != nullptr) CU(cudaMemcpy(info, c->prof_uinfo, sizeof(info), cudaMemcpyDeviceToHost));
        units = (double)info[1];
      }
      w *= units;
    }
    c->prof_n[c->ev_kind[q]] += 1;
    c->prof_ms[c->ev_kind[q]] += ms;
    c->prof_work[c->ev_kind[q]] += w;
  }
  return MVSK_OK;
}

mvsk_status run_pass(mvsk_ctx* c, int prec, int mode, int nin, PassArgs a, const int* live = nullptr,
                     double* spart = nullptr) {
  int stages = 0;
  const size_t smem = rowpass_smem(prec, mode, nin, c->ld, &stages);
  if (smem == 0) return fail(MVSK_EINVAL, "pass (prec %d, mode %d, nin %d) unsupported at ld=%d", prec, mode, nin, c->ld);
  if (prec != P64 && c->Alo == nullptr) return fail(MVSK_EINVAL, "context holds no reduced-precision copy of A");
  a.A = prec == P64 ? (const void*)c->A64 : (const void*)c->Alo;
  a.T = c->T;
  a.ld = c->ld;
  a.part = c->part;
  a.spart = spart != nullptr ? spart : c->spart;
  a.rows_per_cta = c->rows_per_cta;
  a.stages = stages;
  a.err = c->err;
  a.live = live;
  a.counter = c->si + SI_PASSES;
  c->launches += 1;
  static const double esz[] = {8.0, 2.0, 4.0};
  TRY(prof_begin(c, (prec * 16 + mode) * 8 + nin, (double)c->T * (double)c->n * esz[prec]));
  CU(rowpass_launch(prec, mode, nin, a, c->grid, smem, c->stream));
  return prof_end(c);
}

mvsk_status reduce_cols(mvsk_ctx* c, int prec, int nout, double* out, size_t stride, const double* bias, double bscale,
                        const int* skip, const int* live, const double* c1p = nullptr) {
  dim3 g((c->ld + 255) / 256, nout);
  const double sc = 1.0 / (double)c->T;
  c->launches += 1;
  if (prec == P64)
    k_reduce_cols<double><<<g, 256, 0, c->stream>>>((const double*)c->part, c->grid, nout, c->ld, c->n, sc, bias, bscale,
                                                    out, stride, skip, live, c1p);
  else
    k_reduce_cols<float><<<g, 256, 0, c->stream>>>((const float*)c->part, c->grid, nout, c->ld, c->n, sc, bias, bscale, out,
                                                   stride, skip, live, c1p);
  CU(cudaGetLastError());
  return MVSK_OK;
}

// z = A x (FP64), g = -c1 mu + T^-1 A^T psi'(z); scalar partials hold sum psi(z).
mvsk_status pass_valgrad(mvsk_ctx* c, const double* x, double* z, double* g, const int* skip) {
  PassArgs a = pass_args(c);
  a.in[0] = x;
  a.rowout = z;
  a.skip = skip;
  TRY(run_pass(c, P64, M_VALGRAD, 1, a));
  return reduce_cols(c, P64, 1, g, c->ld, c->mu, -c->c[0], skip, nullptr);
}

mvsk_status pass_fwd_z(mvsk_ctx* c, const double* x, double* z) {
  PassArgs a = pass_args(c);
  a.in[0] = x;
  a.rowout = z;
  return run_pass(c, P64, M_FWD, 1, a);
}

mvsk_status pass_ls(mvsk_ctx* c, const double* dir, const int* skip) {
  PassArgs a = pass_args(c);
  a.in[0] = dir;
  a.z = c->in.z;
  a.skip = skip;
  return run_pass(c, P64, M_LS, 1, a);
}

constexpr int kTcCols = 16;  // columns per tensor-core HVP product (one N tile)
mvsk_status ensure_tc_pcg(mvsk_ctx* c);

// Kernel attributes, set once per process before any capture.
mvsk_status init_kernel_attributes() {
  static bool done = false;
  if (done) return MVSK_OK;
  CU(rowpass_init_f64());
  CU(rowpass_init_f32());
  CU(rowpass_init_bf16());
  CU(cudaFuncSetAttribute(k_gemm_tc<128, kTcStages, EpiStoreF64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc_smem_bytes<128>()));
  CU(cudaFuncSetAttribute(k_gemm_tc<kTcCols, 8, EpiPartT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc_smem_bytes<kTcCols, 8>()));
  CU(cudaFuncSetAttribute(k_gemm_tc<64, 6, EpiPartT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc_smem_bytes<64, 6>()));
  CU(cudaFuncSetAttribute(k_gemm_tc<256, 4, EpiPartT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc_smem_bytes<256, 4>()));
  CU(cudaFuncSetAttribute(k_gemm_tc<64, 4, EpiPartT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc_smem_bytes<64, 4>()));
#define MVSK_TC2_ATTR(BN, ST, EPI)                                                                      \
  CU(cudaFuncSetAttribute(k_gemm_tc<BN, ST, EPI, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                          (int)tc_smem_bytes<BN, ST, 2>()))
  MVSK_TC2_ATTR(128, 4, EpiHvp1);
  MVSK_TC2_ATTR(192, 4, EpiHvp1);
  MVSK_TC2_ATTR(256, 3, EpiHvp1);
  MVSK_TC2_ATTR(128, 4, EpiPartT);
  MVSK_TC2_ATTR(192, 4, EpiPartT);
  MVSK_TC2_ATTR(256, 3, EpiPartT);
  MVSK_TC2_ATTR(128, 4, EpiHvp1Tma);
  MVSK_TC2_ATTR(192, 4, EpiHvp1Tma);
  MVSK_TC2_ATTR(256, 3, EpiHvp1Tma);
  MVSK_TC2_ATTR(128, 4, EpiPartTma);
  MVSK_TC2_ATTR(192, 4, EpiPartTma);
  MVSK_TC2_ATTR(256, 3, EpiPartTma);
#undef MVSK_TC2_ATTR
  CU(cudaFuncSetAttribute(k_gemm_tc<16, 8, EpiPartTma>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc_smem_bytes<16, 8>()));
  CU(cudaFuncSetAttribute(k_gemm_tc<64, 4, EpiPartTma>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)tc_smem_bytes<64, 4>()));
  CU(cudaFuncSetAttribute(k_oz_gemm<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes(16)));
  CU(cudaFuncSetAttribute(k_oz_gemm<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes(32)));
  CU(cudaFuncSetAttribute(k_oz_gemm<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes(48)));
  CU(cudaFuncSetAttribute(k_oz_gemm<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes(64)));
  done = true;
  return MVSK_OK;
}
mvsk_status hvp_tc(mvsk_ctx* c, int c0, int nc, const int* skip, const int* live);
mvsk_status third_tc(mvsk_ctx* c, int K, const int* skip);

// ------------------------------------------------ affine-normal block (PCG)
// Sec. 3.2 with the PCG reduced solve: h and the K Hutchinson probes share the
// first PCG round (groups of two columns per pass over A), then
// rhat = K^-1 sum_k (A X_k) o (A p_k), a = P_V T^-1 A^T (psi''' o rhat), a
// second PCG round for H^-1 a, and d = X_h - (||gbar||/m) X_a - nu.
mvsk_status direction_pcg(mvsk_ctx* c) {
  Inst& s = c->in;
  const int K = c->opt.probes;
  const int ncol1 = K + 1;
  const int ca = K + 1;
  const int ngroups = (ncol1 + 1) / 2;
  const int* skipdir = s.si + SI_SKIPDIR;
  const int P = c->dir_prec;
  const int kmax = c->opt.krylov_maxit;
  {
    PassArgs a = pass_args(c);
    a.in[0] = s.nuhat;
    a.in[1] = s.maskF;
    a.z = s.z;
    a.skip = skipdir;
    TRY(run_pass(c, P, M_HVPDIAG, 2, a));
    TRY(reduce_cols(c, P, 2, c->hd, c->ld, nullptr, 0.0, skipdir, nullptr));
  }
  if (K > 0) {
    k_probe_fill<double><<<dim3((c->ld + 255) / 256, K), 256, 0, c->stream>>>(s, K);
    c->launches += 1;
  }
  k_pcg_setup<double><<<1, kVT, 0, c->stream>>>(s, c->spart, c->grid, ngroups);
  CU(cudaGetLastError());
  c->launches += 3 + 2 * kmax;  // setup, setup2, assemble, the pcg_step launches
  if (P == P16 && ncol1 <= kTcCols && 2 * K <= kTcCols) {
    // tensor-core products: every column of a round in one pair of GEMMs
    TRY(ensure_tc_pcg(c));
    for (int it = 0; it < kmax; ++it) {
      TRY(hvp_tc(c, 0, ncol1, skipdir, nullptr));
      k_pcg_step<double><<<ncol1, kPT, 0, c->stream>>>(s, 0, kmax);
      CU(cudaGetLastError());
    }
    if (K > 0) {
      TRY(third_tc(c, K, skipdir));
    } else {
      CU(cudaMemsetAsync(s.at, 0, sizeof(double) * c->ld, c->stream));
    }
    k_pcg_setup2<double><<<1, kVT, 0, c->stream>>>(s, ca, ca / 2);
    CU(cudaGetLastError());
    for (int it = 0; it < kmax; ++it) {
      TRY(hvp_tc(c, ca, 1, skipdir, s.si + SI_LIVE + ca / 2));
      k_pcg_step<double><<<1, kPT, 0, c->stream>>>(s, ca, kmax);
      CU(cudaGetLastError());
    }
    k_assemble<double><<<1, kVT, 0, c->stream>>>(s, ca);
    CU(cudaGetLastError());
    return MVSK_OK;
  }
  for (int it = 0; it < kmax; ++it) {
    for (int g = 0; g < ngroups; ++g) {
      const int c0 = 2 * g;
      const int nin = (c0 + 1 < ncol1) ? 2 : 1;
      PassArgs a = pass_args(c);
      a.in[0] = s.P + (size_t)c0 * c->ld;
      if (nin == 2) a.in[1] = s.P + (size_t)(c0 + 1) * c->ld;
      a.z = s.z;
      a.skip = skipdir;
      TRY(run_pass(c, P, M_HVP, nin, a, s.si + SI_LIVE + g));
      TRY(reduce_cols(c, P, nin, s.Q + (size_t)c0 * c->ld, c->ld, nullptr, 0.0, skipdir, s.si + SI_LIVE + g));
    }
    k_pcg_step<double><<<ncol1, kPT, 0, c->stream>>>(s, 0, kmax);
    CU(cudaGetLastError());
  }
  if (K > 0) {
    for (int k = 0; k < K; ++k) {
      PassArgs a = pass_args(c);
      a.in[0] = s.X + (size_t)(k + 1) * c->ld;
      a.in[1] = s.Bv + (size_t)(k + 1) * c->ld;
      a.rowout = s.rhat;
      a.row_accum = k > 0;
      a.rscale = 1.0 / K;
      a.skip = skipdir;
      TRY(run_pass(c, P, M_RHAT, 2, a));
    }
    PassArgs a = pass_args(c);
    a.z = s.z;
    a.roww = s.rhat;
    a.skip = skipdir;
    TRY(run_pass(c, P, M_BACK, 0, a));
    TRY(reduce_cols(c, P, 1, s.at, c->ld, nullptr, 0.0, skipdir, nullptr));
  } else {
    CU(cudaMemsetAsync(s.at, 0, sizeof(double) * c->ld, c->stream));
  }
  k_pcg_setup2<double><<<1, kVT, 0, c->stream>>>(s, ca, ca / 2);
  CU(cudaGetLastError());
  for (int it = 0; it < kmax; ++it) {
    PassArgs a = pass_args(c);
    a.in[0] = s.P + (size_t)ca * c->ld;
    a.z = s.z;
    a.skip = skipdir;
    TRY(run_pass(c, P, M_HVP, 1, a, s.si + SI_LIVE + ca / 2));
    TRY(reduce_cols(c, P, 1, s.Q + (size_t)ca * c->ld, c->ld, nullptr, 0.0, skipdir, s.si + SI_LIVE + ca / 2));
    k_pcg_step<double><<<1, kPT, 0, c->stream>>>(s, ca, kmax);
    CU(cudaGetLastError());
  }
  k_assemble<double><<<1, kVT, 0, c->stream>>>(s, ca);
  CU(cudaGetLastError());
  return MVSK_OK;
}

mvsk_status read_ints(mvsk_ctx* c, int* dst, int first, int count);

// ------------------------------------------------ tensor-core helpers
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D BF16 tensor map over a row-major (outer x inner) array with 128-byte swizzle.
mvsk_status make_tmap_bf16(CUtensorMap* tm, const void* base, unsigned long long inner, unsigned long long outer,
                           unsigned long long row_bytes, unsigned box_inner, unsigned box_outer) {
  auto enc = tmap_encoder();
  if (enc == nullptr) return fail(MVSK_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (row_bytes & 15) != 0)
    return fail(MVSK_EINVAL, "tensor map base/stride not 16-byte aligned");
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(MVSK_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return MVSK_OK;
}

// Tensor map for the bulk tensor stores of the GEMM epilogues (no swizzle):
// rank 2 or 3, dims[0] innermost, strides in bytes for dims 1.., box in elements.
mvsk_status make_tmap_store(CUtensorMap* tm, CUtensorMapDataType dt, int rank, const void* base,
                            const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box) {
  auto enc = tmap_encoder();
  if (enc == nullptr) return fail(MVSK_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return fail(MVSK_EINVAL, "tensor map base not 16-byte aligned");
  for (int i = 0; i + 1 < rank; ++i)
    if ((strides[i] & 15) != 0) return fail(MVSK_EINVAL, "tensor map stride not a multiple of 16 bytes");
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(tm, dt, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(MVSK_ECUDA, "cuTensorMapEncodeTiled (store) failed (%d)", (int)r);
  return MVSK_OK;
}

// out[j*ldo + t] = bf16(sc_t * A[t*lda + j]) for j < n, t < T; zero for T <= t < Tp.
__global__ void k_transpose_bf16(const double* A, int lda, long long T, int n, const double* sc, __nv_bfloat16* out,
                                 long long ldo, long long Tp) {
  __shared__ float tile[32][33];
  const long long t0 = (long long)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const long long t = t0 + threadIdx.y + 8 * k;
    const int j = j0 + threadIdx.x;
    double v = 0.0;
    if (t < T && j < n) v = A[(size_t)t * lda + j] * (sc != nullptr ? sc[t] : 1.0);
    tile[threadIdx.y + 8 * k][threadIdx.x] = (float)v;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = j0 + threadIdx.y + 8 * k;
    const long long t = t0 + threadIdx.x;
    if (j < n && t < Tp) out[(size_t)j * ldo + t] = __float2bfloat16(tile[threadIdx.x][threadIdx.y + 8 * k]);
  }
}

mvsk_status transpose_bf16(mvsk_ctx* c, const double* sc, __nv_bfloat16* out) {
  dim3 g((unsigned)((c->Tp + 31) / 32), (unsigned)((c->n + 31) / 32));
  k_transpose_bf16<<<g, dim3(32, 8), 0, c->stream>>>(c->A64, c->ld, c->T, c->n, sc, out, c->Tp, c->Tp);
  c->launches += 1;
  CU(cudaGetLastError());
  return MVSK_OK;
}

mvsk_status ensure_tc_operands(mvsk_ctx* c) {
  if (c->A16T != nullptr) return MVSK_OK;
  c->Tp = (c->T + 7) / 8 * 8;
  void* p;
  TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * (size_t)c->n * c->Tp));
  c->A16T = (__nv_bfloat16*)p;
  TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * (size_t)c->n * c->Tp));
  c->W16T = (__nv_bfloat16*)p;
  return transpose_bf16(c, nullptr, c->A16T);
}

// C (M x N, FP64, ldc) = alpha * A B^T with A (M x K) and B (N x K) K-major BF16 (row bytes rb).
mvsk_status gemm_tc_f64(mvsk_ctx* c, const __nv_bfloat16* A, int M, const __nv_bfloat16* B, int N, long long K,
                        long long ldk, double alpha, double* C, long long ldc) {
  CUtensorMap ta, tb;
  TRY(make_tmap_bf16(&ta, A, (unsigned long long)ldk, (unsigned long long)M, (unsigned long long)ldk * 2, kTcBK, kTcBM));
  TRY(make_tmap_bf16(&tb, B, (unsigned long long)ldk, (unsigned long long)N, (unsigned long long)ldk * 2, kTcBK, 128));
  auto kern = k_gemm_tc<128, kTcStages, EpiStoreF64>;
  const size_t smem = tc_smem_bytes<128>();
  EpiStoreF64 epi{C, ldc, alpha, M, N};
  dim3 grid((unsigned)((N + 127) / 128), (unsigned)((M + kTcBM - 1) / kTcBM), 1);
  const int nk = (int)((K + kTcBK - 1) / kTcBK);
  kern<<<grid, 128, smem, c->stream>>>(ta, tb, M, N, (int)K, nk, epi, c->err, nullptr, nullptr, nullptr);
  c->launches += 1;
  CU(cudaGetLastError());
  return MVSK_OK;
}

// ------------------------------------------------ tensor-core PCG products

// dst[j][i] = bf16(src_j[i]) for j < nc, i < ld; columns come from up to two strided sources
__global__ void k_cols_bf16(const double* srcA, const double* srcB, int nc, int interleave, int ld, __nv_bfloat16* dst,
                            const int* skip) {
  if (skip != nullptr && *skip != 0) return;
  const long long tot = (long long)nc * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / ld), i = (int)(e % ld);
    double v;
    if (interleave) v = (j & 1) ? srcB[(size_t)(j >> 1) * ld + i] : srcA[(size_t)(j >> 1) * ld + i];
    else v = srcA[(size_t)j * ld + i];
    dst[e] = __float2bfloat16((float)v);
  }
}

// S^T[j][t] = bf16(psi''(z_t) * sum_z part[z][j][t]) (t < T; padding t < Tp stays zero)
__global__ void k_reduce_hvp1(const float* part, int splits, int nc, long long T, long long ldp, const double* z,
                              double c2, double c3, double c4, __nv_bfloat16* S, long long Tp, const int* skip) {
  if (skip != nullptr && *skip != 0) return;
  const Psi psi{c2, c3, c4};
  const long long tot = (long long)nc * T;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / T);
    const long long t = e % T;
    float acc = 0.f;
    for (int q = 0; q < splits; ++q) acc += part[((size_t)q * nc + j) * ldp + t];
    S[(size_t)j * Tp + t] = __float2bfloat16((float)(psi.d2(z[t]) * (double)acc));
  }
}

// Q[j][i] = scale * sum_z part[z][j][i] for i < n, 0 for n <= i < ld
__global__ void k_reduce_hvp2(const float* part, int splits, int nc, int n, int ld, long long ldp, double scale,
                              double* Q, const int* skip) {
  if (skip != nullptr && *skip != 0) return;
  const long long tot = (long long)nc * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / ld), i = (int)(e % ld);
    double acc = 0.0;
    if (i < n)
      for (int q = 0; q < splits; ++q) acc += (double)part[((size_t)q * nc + j) * ldp + i];
    Q[(size_t)j * ld + i] = scale * acc;
  }
}

// rhat[t] = K^-1 sum_k (A X_k)_t (A p_k)_t from the interleaved product columns
__global__ void k_reduce_rhat(const float* part, int splits, int nc, long long T, long long ldp, double* rhat,
                              const int* skip) {
  if (skip != nullptr && *skip != 0) return;
  const int K = nc / 2;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (long long)gridDim.x * blockDim.x) {
    double r = 0.0;
    for (int k = 0; k < K; ++k) {
      float u = 0.f, v = 0.f;
      for (int q = 0; q < splits; ++q) {
        u += part[((size_t)q * nc + 2 * k) * ldp + t];
        v += part[((size_t)q * nc + 2 * k + 1) * ldp + t];
      }
      r += (double)u * (double)v;
    }
    rhat[t] = r / K;
  }
}

// S^T[0][t] = bf16(psi3(z_t) rhat_t), psi3 the third derivative of psi
__global__ void k_back_weights(const double* z, const double* rhat, long long T, double c3, double c4,
                               __nv_bfloat16* S, const int* skip) {
  if (skip != nullptr && *skip != 0) return;
  const Psi psi{0.0, c3, c4};
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (long long)gridDim.x * blockDim.x)
    S[t] = __float2bfloat16((float)(psi.d3(z[t]) * rhat[t]));
}

mvsk_status ensure_tc_pcg(mvsk_ctx* c) {
  if (c->P16 != nullptr) return MVSK_OK;
  TRY(ensure_tc_operands(c));
  void* p;
  TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * (size_t)kTcCols * c->ld));
  c->P16 = (__nv_bfloat16*)p;
  TRY(dalloc(c, &p, sizeof(__nv_bfloat16) * (size_t)kTcCols * c->Tp));
  c->S16T = (__nv_bfloat16*)p;
  const size_t np = (size_t)8 * kTcCols * (size_t)(c->T > c->ld ? c->T : c->ld);
  TRY(dalloc(c, &p, sizeof(float) * np));
  c->part32 = (float*)p;
  TRY(make_tmap_bf16(&c->tm_A16, c->Alo, (unsigned long long)c->ld, (unsigned long long)c->T,
                     (unsigned long long)c->ld * 2, kTcBK, kTcBM));
  TRY(make_tmap_bf16(&c->tm_P16, c->P16, (unsigned long long)c->ld, kTcCols, (unsigned long long)c->ld * 2, kTcBK,
                     kTcCols));
  TRY(make_tmap_bf16(&c->tm_A16T, c->A16T, (unsigned long long)c->Tp, (unsigned long long)c->n,
                     (unsigned long long)c->Tp * 2, kTcBK, kTcBM));
  TRY(make_tmap_bf16(&c->tm_S16T, c->S16T, (unsigned long long)c->Tp, kTcCols, (unsigned long long)c->Tp * 2, kTcBK,
                     kTcCols));
  return MVSK_OK;
}

// Split-K launch of a 128 x 16 tensor-core product writing FP32 partials; returns the split count.
mvsk_status tc_partials(mvsk_ctx* c, const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, long long K,
                        long long ldp, const int* skip, const int* live, int* splits_out) {
  auto kern = k_gemm_tc<kTcCols, 8, EpiPartT>;
  const size_t smem = tc_smem_bytes<kTcCols, 8>();
  const int mt = (M + kTcBM - 1) / kTcBM;
  const int nk = (int)((K + kTcBK - 1) / kTcBK);
  int want = (2 * c->nsm + mt - 1) / mt;
  if (want > 8) want = 8;
  if (want > nk) want = nk;
  if (want < 1) want = 1;
  const int ktps = (nk + want - 1) / want;
  const int splits = (nk + ktps - 1) / ktps;
  EpiPartT epi{c->part32, ldp, M, N};
  dim3 grid(1, (unsigned)mt, (unsigned)splits);
  kern<<<grid, 128, smem, c->stream>>>(ta, tb, M, N, (int)K, ktps, epi, c->err, skip, live, nullptr);
  c->launches += 1;
  CU(cudaGetLastError());
  *splits_out = splits;
  return MVSK_OK;
}

// Q[c0 .. c0+nc) = T^-1 A^T (psi''(z) o A P[c0 .. c0+nc)) on the tensor cores (BF16 A, FP32 accumulate).
mvsk_status hvp_tc(mvsk_ctx* c, int c0, int nc, const int* skip, const int* live) {
  Inst& s = c->in;
  const int ld = c->ld;
  const int gb = 2 * c->nsm;
  k_cols_bf16<<<gb, 256, 0, c->stream>>>(s.P + (size_t)c0 * ld, nullptr, nc, 0, ld, c->P16, skip);
  int s1 = 0, s2 = 0;
  TRY(tc_partials(c, c->tm_A16, c->tm_P16, (int)c->T, nc, ld, c->T, skip, live, &s1));
  k_reduce_hvp1<<<gb, 256, 0, c->stream>>>(c->part32, s1, nc, c->T, c->T, s.z, c->c[1], c->c[2], c->c[3], c->S16T,
                                           c->Tp, skip);
  TRY(tc_partials(c, c->tm_A16T, c->tm_S16T, c->n, nc, c->Tp, ld, skip, live, &s2));
  k_reduce_hvp2<<<gb, 256, 0, c->stream>>>(c->part32, s2, nc, c->n, ld, ld, 1.0 / (double)c->T,
                                           s.Q + (size_t)c0 * ld, skip);
  c->launches += 3;
  CU(cudaGetLastError());
  return MVSK_OK;
}

// rhat and a = T^-1 A^T (psi3(z) o rhat) on the tensor cores.
mvsk_status third_tc(mvsk_ctx* c, int K, const int* skip) {
  Inst& s = c->in;
  const int ld = c->ld;
  const int gb = 2 * c->nsm;
  k_cols_bf16<<<gb, 256, 0, c->stream>>>(s.X + ld, s.Bv + ld, 2 * K, 1, ld, c->P16, skip);
  int s1 = 0, s2 = 0;
  TRY(tc_partials(c, c->tm_A16, c->tm_P16, (int)c->T, 2 * K, ld, c->T, skip, nullptr, &s1));
  k_reduce_rhat<<<gb, 256, 0, c->stream>>>(c->part32, s1, 2 * K, c->T, c->T, s.rhat, skip);
  k_back_weights<<<gb, 256, 0, c->stream>>>(s.z, s.rhat, c->T, c->c[2], c->c[3], c->S16T, skip);
  TRY(tc_partials(c, c->tm_A16T, c->tm_S16T, c->n, 1, c->Tp, ld, skip, nullptr, &s2));
  k_reduce_hvp2<<<gb, 256, 0, c->stream>>>(c->part32, s2, 1, c->n, ld, ld, 1.0 / (double)c->T, s.at, skip);
  c->launches += 4;
  CU(cudaGetLastError());
  return MVSK_OK;
}

#include "direct_impl.cuh"
#include "ozaki_impl.cuh"
#include "batch_impl.cuh"

mvsk_status direction(mvsk_ctx* c, int cfg) { return cfg == MVSK_PCG ? direction_pcg(c) : direction_direct(c); }

// One iteration of Alg. 1: oracle block, affine-normal block, quartic step, boundary block.
mvsk_status launch_iteration(mvsk_ctx* c, int cfg) {
  Inst& s = c->in;
  const int* done = s.si + SI_DONE;
  TRY(pass_valgrad(c, s.x, s.z, s.g, done));
  k_face<<<1, kVT, 0, c->stream>>>(s, c->spart, c->grid);
  CU(cudaGetLastError());
  c->launches += 5;  // k_face, k_decide1, k_decide2, k_end_iter (+1 below)
  TRY(direction(c, cfg));
  TRY(pass_ls(c, s.d, done));
  k_decide1<<<1, kVT, 0, c->stream>>>(s, c->spart, c->grid, nullptr);
  CU(cudaGetLastError());
  TRY(pass_ls(c, s.dstep, s.si + SI_SKIPLS));
  k_decide2<<<1, kVT, 0, c->stream>>>(s, c->spart, c->grid);
  CU(cudaGetLastError());
  k_end_iter<<<1, 32, 0, c->stream>>>(s);
  CU(cudaGetLastError());
  return MVSK_OK;
}

// Host copies of a few device ints / doubles.
mvsk_status read_ints(mvsk_ctx* c, int* dst, int first, int count) {
  CU(cudaMemcpyAsync(dst, c->si + first, sizeof(int) * count, cudaMemcpyDeviceToHost, c->stream));
  TRY(sync(c));
  return MVSK_OK;
}

mvsk_status init_state(mvsk_ctx* c, int cfg, double tol, const double cc[4]) {
  const Options& o = c->opt;
  const bool pcg = cfg == MVSK_PCG;
  const double reg = isnan(o.reg) ? (pcg ? 1e-4 : 0.0) : o.reg;
  double h[12] = {o.tau, o.eps_act, o.release_ratio, reg, o.krylov_tol, cc[0], cc[1], cc[2], cc[3],
                  1.0 / (double)c->T, o.descent_eps, o.stall_factor};
  double* dopts = c->vec_scratch;  // 12 doubles
  CU(cudaMemcpyAsync(dopts, h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  k_init_state<<<1, 32, 0, c->stream>>>(c->in, tol, o.eta, pcg ? o.pcg_max_iter : o.max_iter, pcg ? 1 : 0,
                                        o.stall_window, o.probes, o.probe_seed, o.krylov_maxit, o.arc_halvings,
                                        o.line_search, dopts);
  CU(cudaGetLastError());
  return MVSK_OK;
}

void set_coefs(mvsk_ctx* c, const double cc[4]) {
  for (int q = 0; q < 4; ++q) c->c[q] = cc[q];
}

struct SolveOut {
  int status = MVSK_OK;
  int iters = 0, restarts = 0;
};

// Plain YAND-MVSK solve of one instance with coefficients cc (Alg. 1 plus the
// stall-recovery phases of the PCG configuration).  Result in c->in.x.
mvsk_status solve_instance(mvsk_ctx* c, int cfg, double tol, const double* w0_dev, const double cc[4], SolveOut* so,
                           std::chrono::steady_clock::time_point t0) {
  Inst& s = c->in;
  set_coefs(c, cc);
  TRY(init_state(c, cfg, tol, cc));
  // kkt at x0 = 1/n (denominator of kkt_rel)
  k_fill<<<(c->ld + 255) / 256, 256, 0, c->stream>>>(s.x, c->n, c->ld, 1.0 / c->n);
  TRY(pass_valgrad(c, s.x, s.z, s.g, nullptr));
  k_kkt0<<<1, kVT, 0, c->stream>>>(s);
  CU(cudaGetLastError());
  if (w0_dev != nullptr) CU(cudaMemcpyAsync(s.x, w0_dev, sizeof(double) * c->ld, cudaMemcpyDeviceToDevice, c->stream));
  if (c->n == 1) {
    so->status = MVSK_OK;
    return MVSK_OK;
  }
  const Options& o = c->opt;
  struct Phase {
    double eta;
    int maxit;
  };
  std::vector<Phase> phases;
  if (cfg == MVSK_PCG) {
    phases = {{o.eta, o.pcg_max_iter}, {o.restart_eta1, o.restart_iter1}, {o.restart_eta2, o.restart_iter2}};
  } else {
    phases = {{o.eta, o.max_iter}};
  }
  int done = 0;
  so->status = MVSK_ENOTCONVERGED;
  // The PCG iteration is driven entirely by device flags: capture it once as a
  // CUDA graph and replay it (three replays between host checks of the flag).
  cudaGraphExec_t gexec = nullptr;
  long long per_graph = 0;
  const bool graph = cfg == MVSK_PCG && c->use_graphs && !o.trace;
  if (graph) {
    if (c->dir_prec == P16) TRY(ensure_tc_pcg(c));
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const long long l0 = c->launches;
    c->ev_graph_begin = c->ev_kind.size();
    const mvsk_status cs = launch_iteration(c, cfg);
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
  const int every = graph ? 3 : 1;
  for (size_t ph = 0; ph < phases.size(); ++ph) {
    if (ph > 0) so->restarts += 1;
    k_new_phase<<<1, 32, 0, c->stream>>>(s, phases[ph].eta, phases[ph].maxit,
                                         ph + 1 < phases.size() ? o.stall_window : 0);
    CU(cudaGetLastError());
    for (int it = 0; it <= phases[ph].maxit; ++it) {
      if (graph) {
        CU(cudaGraphLaunch(gexec, c->stream));
        c->launches += per_graph;
        if (c->prof_on) {
          CU(cudaStreamSynchronize(c->stream));
          TRY(prof_collect(c, c->ev_graph_begin, c->ev_graph_end));
        }
        if ((it % every) != every - 1 && it != phases[ph].maxit) continue;
      } else {
        TRY(launch_iteration(c, cfg));
      }
      TRY(read_ints(c, &done, SI_DONE, 1));
      if (o.trace) {
        int hi[kSI];
        double hd[kSD];
        CU(cudaMemcpy(hi, s.si, sizeof(hi), cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(hd, s.sd, sizeof(hd), cudaMemcpyDeviceToHost));
        fprintf(stderr,
                "[mvsk] phase %zu it %d done %d kkt_rel %.3e f %.12e m %d gn %.3e branch %d amax %.3e eta_k %.3e "
                "alpha %.3e lam %.3e kry %d\n",
                ph, hi[SI_ITER], hi[SI_DONE], hd[SD_KKTREL], hd[SD_F], hi[SI_M], hd[SD_GN], hi[SI_BRANCH],
                hd[SD_AMAX], hd[SD_ETAK], hd[SD_ALPHA], hd[SD_LAM], hi[SI_KRY]);
      }
      if (done != 0) break;
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > o.max_elapsed) {
        so->status = MVSK_ETIMEOUT;
        done = 4;
        break;
      }
    }
    if (done == 1) {
      so->status = MVSK_OK;
      break;
    }
    if (done == 3) {
      so->status = MVSK_ENUMERIC;
      break;
    }
    if (done == 4) break;
  }
  if (so->status != MVSK_OK)
    CU(cudaMemcpyAsync(s.x, s.bestx, sizeof(double) * c->ld, cudaMemcpyDeviceToDevice, c->stream));
  return MVSK_OK;
}

// f, kkt and mu^T x at c->in.x with the current coefficients.
mvsk_status eval_here(mvsk_ctx* c, double out3[3]) {
  Inst& s = c->in;
  TRY(pass_valgrad(c, s.x, s.z, s.g, nullptr));
  double* d3 = c->vec_scratch + 16;
  k_eval_finish<<<1, kVT, 0, c->stream>>>(s, c->spart, c->grid, d3);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(out3, d3, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TRY(sync(c));
  return MVSK_OK;
}

// Solve with optional return-target calibration of c1 (Illinois regula falsi
// on mu^T x*(c1) = target; Sec. 6).  Result in c->in.x; fills info.
mvsk_status solve_with_target(mvsk_ctx* c, int cfg, double tol, const double* w0_dev, const double lam[4],
                              double target, mvsk_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  double cc[4];
  const double s = c->s_equal;
  if (c->opt.pref_scaling == 1 && s > 0.0 && isfinite(s)) {
    cc[0] = lam[0] / s;
    cc[1] = lam[1] / (s * s);
    cc[2] = lam[2] / (s * s * s);
    cc[3] = lam[3] / (s * s * s * s);
  } else {
    for (int q = 0; q < 4; ++q) cc[q] = lam[q];
  }
  Inst& in = c->in;
  const size_t vb = sizeof(double) * c->ld;
  double* xlo = in.tmp + (size_t)20 * c->ld;
  double* xhi = xlo + c->ld;
  int evals = 0, iters = 0, restarts = 0, last_it = -1;
  SolveOut so;
  double ev[3];
  auto run = [&](double c1, const double* w0, double* h) -> mvsk_status {
    double c4[4] = {c1, cc[1], cc[2], cc[3]};
    SolveOut o;
    TRY(solve_instance(c, cfg, tol, w0, c4, &o, t0));
    int it = 0;
    TRY(read_ints(c, &it, SI_ITER, 1));
    iters += it;
    last_it = it;
    restarts += o.restarts;
    so = o;
    evals += 1;
    TRY(eval_here(c, ev));
    *h = ev[2] - target;
    return MVSK_OK;
  };
  double h = 0.0;
  if (isnan(target)) {
    TRY(run(cc[0], w0_dev, &h));
  } else {
    const double scale = c->mu_absmax;
    const double gap_tol = c->opt.cal_rel_tol * scale;
    const double c1_ref = fmax(cc[1], 1e-300) * s * s / fmax(scale, 1e-300);
    const double c1_max = 1e6 * c1_ref;
    double h_lo, h_hi, c_lo = 0.0, c_hi;
    TRY(run(0.0, nullptr, &h_lo));
    cc[0] = 0.0;
    if (!(h_lo >= -gap_tol)) {
      CU(cudaMemcpyAsync(xlo, in.x, vb, cudaMemcpyDeviceToDevice, c->stream));
      const double c1_start = c->opt.pref_scaling == 1 && s > 0.0 && isfinite(s) ? lam[0] / s : lam[0];
      c_hi = c1_start > 0.0 ? c1_start : c1_ref;
      TRY(run(c_hi, xlo, &h_hi));
      CU(cudaMemcpyAsync(xhi, in.x, vb, cudaMemcpyDeviceToDevice, c->stream));
      while (h_hi < 0.0 && c_hi < c1_max) {
        c_lo = c_hi;
        h_lo = h_hi;
        CU(cudaMemcpyAsync(xlo, xhi, vb, cudaMemcpyDeviceToDevice, c->stream));
        c_hi = fmin(8.0 * c_hi, c1_max);
        TRY(run(c_hi, xlo, &h_hi));
        CU(cudaMemcpyAsync(xhi, in.x, vb, cudaMemcpyDeviceToDevice, c->stream));
      }
      cc[0] = c_hi;
      if (h_hi >= 0.0 && !(fabs(h_hi) <= gap_tol)) {
        int side = 0;
        while (evals < c->opt.cal_max_evals) {
          double cm = c_hi - h_hi * (c_hi - c_lo) / (h_hi - h_lo);
          if (!(c_lo < cm && cm < c_hi)) cm = 0.5 * (c_lo + c_hi);
          const double* w0 = (cm - c_lo) <= (c_hi - cm) ? xlo : xhi;
          double hm;
          TRY(run(cm, w0, &hm));
          cc[0] = cm;
          // a solve that needed no iteration from its warm start resolves the
          // mean no finer: its point ends the calibration near the target
          if (fabs(hm) <= gap_tol || (last_it == 0 && fabs(hm) <= 10.0 * gap_tol) ||
              (c_hi - c_lo) <= c->opt.cal_bracket_tol * c_hi)
            break;
          if (hm < 0.0) {
            c_lo = cm;
            h_lo = hm;
            CU(cudaMemcpyAsync(xlo, in.x, vb, cudaMemcpyDeviceToDevice, c->stream));
            if (side == -1) h_hi *= 0.5;
            side = -1;
          } else {
            c_hi = cm;
            h_hi = hm;
            CU(cudaMemcpyAsync(xhi, in.x, vb, cudaMemcpyDeviceToDevice, c->stream));
            if (side == 1) h_lo *= 0.5;
            side = 1;
          }
          cc[0] = c_hi;
          if (evals >= c->opt.cal_max_evals) {
            CU(cudaMemcpyAsync(in.x, xhi, vb, cudaMemcpyDeviceToDevice, c->stream));
            double c4[4] = {c_hi, cc[1], cc[2], cc[3]};
            set_coefs(c, c4);
            TRY(eval_here(c, ev));
          }
        }
      }
    }
  }
  if (info != nullptr) {
    int cnt[kSI];
    CU(cudaMemcpyAsync(cnt, c->si, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    TRY(sync(c));
    // kkt_rel against kkt(1/n): sd[SD_KKT0] of the last solve
    double k0 = 0.0;
    CU(cudaMemcpy(&k0, in.sd + SD_KKT0, sizeof(double), cudaMemcpyDeviceToHost));
    memset(info, 0, sizeof(*info));
    info->iters = iters;
    info->restarts = restarts;
    info->passes = cnt[SI_PASSES];
    info->krylov_iters = cnt[SI_KRY];
    info->third_calls = cnt[SI_THIRD];
    info->evals = evals;
    info->f = ev[0];
    info->kkt_residual = ev[1];
    info->kkt0 = k0;
    info->kkt_rel = c->n == 1 ? 0.0 : ev[1] / fmax(k0, 1e-300);
    for (int q = 0; q < 4; ++q) info->c[q] = c->c[q];
    info->achieved_mean = ev[2];
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->status = so.status;
    std::vector<double> hx(c->n);
    CU(cudaMemcpy(hx.data(), in.x, sizeof(double) * c->n, cudaMemcpyDeviceToHost));
    int fc = 0;
    for (int i = 0; i < c->n; ++i) fc += (hx[i] - c->opt.tau > c->opt.eps_act);
    info->free_count = fc;
  }
  return (mvsk_status)so.status;
}

mvsk_status check_w0(mvsk_ctx* c, const double* w0, double* dst) {
  std::vector<double> h(c->n);
  CU(cudaMemcpy(h.data(), w0, sizeof(double) * c->n, cudaMemcpyDefault));
  double s = 0.0, mn = INFINITY;
  for (int i = 0; i < c->n; ++i) {
    if (!isfinite(h[i])) return fail(MVSK_EINVAL, "w0[%d] is not finite", i);
    s += h[i];
    mn = fmin(mn, h[i]);
  }
  if (fabs(s - 1.0) > 1e-9 || mn < c->opt.tau * (1.0 - 1e-9))
    return fail(MVSK_EINVAL, "w0 is not in Delta(tau): sum %.17g, min %.3g", s, mn);
  CU(cudaMemsetAsync(dst, 0, sizeof(double) * c->ld, c->stream));
  CU(cudaMemcpyAsync(dst, h.data(), sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream));
  TRY(sync(c));
  return MVSK_OK;
}

mvsk_status equal_weight_scale(mvsk_ctx* c) {
  Inst& s = c->in;
  k_fill<<<(c->ld + 255) / 256, 256, 0, c->stream>>>(s.x, c->n, c->ld, 1.0 / c->n);
  TRY(pass_fwd_z(c, s.x, s.z));
  double* d = c->vec_scratch + 24;
  k_sumsq<<<1, kVT, 0, c->stream>>>(s.z, c->T, d);
  double h = 0.0;
  CU(cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TRY(sync(c));
  c->s_equal = sqrt(h / (double)c->T);
  return MVSK_OK;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

mvsk_status mvsk_create(const double* R, int64_t T, int64_t n, int64_t ld, uint32_t flags, mvsk_ctx** out) {
  if (out == nullptr || R == nullptr) return fail(MVSK_EINVAL, "null argument");
  *out = nullptr;
  if (T < 1 || n < 1 || n > kMaxCols || ld < n) return fail(MVSK_EINVAL, "bad sizes T=%lld n=%lld ld=%lld", (long long)T, (long long)n, (long long)ld);
  if (flags > MVSK_PREC_MIXED_FP32) return fail(MVSK_EINVAL, "unknown flags %u", flags);
  mvsk_ctx* c = new (std::nothrow) mvsk_ctx();
  if (c == nullptr) return fail(MVSK_ENOMEM, "host allocation failed");
  auto bail = [&](mvsk_status st_) {
    mvsk_destroy(c);
    return st_;
  };
  mvsk_status st;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return bail(fail(MVSK_ECUDA, "no CUDA device"));
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return bail(fail(MVSK_ECUDA, "cudaGetDeviceProperties failed"));
  c->nsm = prop.multiProcessorCount;
  if (cudaStreamCreate(&c->own_stream) != cudaSuccess) return bail(fail(MVSK_ECUDA, "cudaStreamCreate failed"));
  c->stream = c->own_stream;
  if ((st = init_kernel_attributes()) != MVSK_OK) return bail(st);
  c->T = T;
  c->n = (int)n;
  c->ld = (int)((n + kPad - 1) / kPad * kPad);
  c->flags = flags;
  c->dir_prec = flags == MVSK_PREC_MIXED_BF16 ? P16 : (flags == MVSK_PREC_MIXED_FP32 ? P32 : P64);
  c->grid = (int)(T < c->nsm ? T : c->nsm);
  c->rows_per_cta = (int)((T + c->grid - 1) / c->grid);
  c->grid = (int)((T + c->rows_per_cta - 1) / c->rows_per_cta);
  const size_t ldb = sizeof(double) * c->ld;
#define ALLOC(ptr, bytes)                                              \
  do {                                                                 \
    void* p_ = nullptr;                                                \
    if ((st = dalloc(c, &p_, (bytes))) != MVSK_OK) return bail(st);    \
    ptr = reinterpret_cast<decltype(ptr)>(p_);                         \
  } while (0)
  ALLOC(c->A64, ldb * (size_t)T);
  if (flags == MVSK_PREC_MIXED_BF16) ALLOC(c->Alo, sizeof(__nv_bfloat16) * c->ld * (size_t)T);
  if (flags == MVSK_PREC_MIXED_FP32) ALLOC(c->Alo, sizeof(float) * c->ld * (size_t)T);
  ALLOC(c->mu, ldb);
  ALLOC(c->err, 64);
  if (cudaMallocHost(&c->hword, 64) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(MVSK_ENOMEM, "pinned host word allocation failed"));
  }
  if (cudaMemcpy2DAsync(c->A64, ldb, R, sizeof(double) * ld, sizeof(double) * n, T, cudaMemcpyDefault, c->stream) !=
      cudaSuccess)
    return bail(fail(MVSK_ECUDA, "copy of R failed"));
  k_colmean<<<(c->n + 127) / 128, 128, 0, c->stream>>>(c->A64, T, c->n, c->ld, c->mu);
  const int cg = 4 * c->nsm;
  if (flags == MVSK_PREC_MIXED_BF16)
    k_centre<__nv_bfloat16><<<cg, 256, 0, c->stream>>>(c->A64, (__nv_bfloat16*)c->Alo, T, c->n, c->ld, c->mu, c->err);
  else if (flags == MVSK_PREC_MIXED_FP32)
    k_centre<float><<<cg, 256, 0, c->stream>>>(c->A64, (float*)c->Alo, T, c->n, c->ld, c->mu, c->err);
  else
    k_centre<float><<<cg, 256, 0, c->stream>>>(c->A64, (float*)nullptr, T, c->n, c->ld, c->mu, c->err);
  if (cudaGetLastError() != cudaSuccess) return bail(fail(MVSK_ECUDA, "centring launch failed"));
  int bad = 0;
  if (cudaMemcpy(&bad, c->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return bail(fail(MVSK_ECUDA, "sync failed"));
  if (bad) return bail(fail(MVSK_EINVAL, "R holds a non-finite value"));
  // instance state and workspace
  Inst& s = c->in;
  c->ncolmax = 20;
  ALLOC(c->sd, sizeof(double) * kSD);
  ALLOC(c->si, sizeof(int) * kSI);
  s.sd = c->sd;
  s.si = c->si;
  s.mu = c->mu;
  ALLOC(s.x, ldb);
  ALLOC(s.g, ldb);
  ALLOC(s.nuhat, ldb);
  ALLOC(s.maskF, ldb);
  ALLOC(s.d, ldb);
  ALLOC(s.dstep, ldb);
  ALLOC(s.xbar, ldb);
  ALLOC(s.at, ldb);
  ALLOC(s.bestx, ldb);
  ALLOC(s.tmp, ldb * (size_t)(c->ncolmax + 4));
  ALLOC(c->hd, 2 * ldb);
  s.Gnu = c->hd;
  s.diagG = c->hd + c->ld;
  ALLOC(s.z, sizeof(double) * (size_t)T);
  ALLOC(s.rhat, sizeof(double) * (size_t)T);
  ALLOC(s.X, ldb * c->ncolmax);
  ALLOC(s.R, ldb * c->ncolmax);
  ALLOC(s.Zc, ldb * c->ncolmax);
  ALLOC(s.P, ldb * c->ncolmax);
  ALLOC(s.Q, ldb * c->ncolmax);
  ALLOC(s.Bv, ldb * c->ncolmax);
  ALLOC(s.rz, sizeof(double) * c->ncolmax);
  ALLOC(s.rhsn, sizeof(double) * c->ncolmax);
  ALLOC(c->part, sizeof(double) * 2 * (size_t)c->ld * c->grid);
  ALLOC(c->spart, sizeof(double) * 16 * (size_t)c->grid);
  ALLOC(c->fwd, sizeof(double) * 4 * (size_t)T);
  ALLOC(c->vec_scratch, sizeof(double) * (64 + 4 * (size_t)c->ld));
  s.n = c->n;
  s.ld = c->ld;
  s.T = T;
  s.spart = c->spart;
  s.vs = c->ld;
  s.ts = T;
  s.cs = (long long)c->ld * c->ncolmax;
  s.ps = (long long)c->ld * (c->ncolmax + 4);
  s.ncs = c->ncolmax;
  s.ss = 16LL * c->grid;
#undef ALLOC
  std::vector<double> hmu(c->n);
  if (cudaMemcpy(hmu.data(), c->mu, sizeof(double) * c->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return bail(fail(MVSK_ECUDA, "copy of mu failed"));
  for (int i = 0; i < c->n; ++i) c->mu_absmax = fmax(c->mu_absmax, fabs(hmu[i]));
  if ((st = equal_weight_scale(c)) != MVSK_OK) return bail(st);
  *out = c;
  return MVSK_OK;
}

mvsk_status mvsk_set_stream(mvsk_ctx* c, void* stream) {
  if (c == nullptr) return fail(MVSK_EINVAL, "null context");
  c->stream = stream != nullptr ? (cudaStream_t)stream : c->own_stream;
  return MVSK_OK;
}

mvsk_status mvsk_set_prefs(mvsk_ctx* c, const double lambda[4], double target) {
  if (c == nullptr || lambda == nullptr) return fail(MVSK_EINVAL, "null argument");
  for (int q = 0; q < 4; ++q)
    if (!(lambda[q] >= 0.0) || !isfinite(lambda[q])) return fail(MVSK_EINVAL, "lambda[%d] must be finite and >= 0", q);
  if (isinf(target)) return fail(MVSK_EINVAL, "target must be finite or NaN");
  for (int q = 0; q < 4; ++q) c->lam[q] = lambda[q];
  c->target = target;
  const double s = c->s_equal;
  const bool stdz = c->opt.pref_scaling == 1 && s > 0.0 && isfinite(s);
  for (int q = 0; q < 4; ++q) c->c[q] = stdz ? lambda[q] / pow(s, q + 1) : lambda[q];
  c->prefs_set = true;
  return MVSK_OK;
}

mvsk_status mvsk_set_option(mvsk_ctx* c, const char* key, double v) {
  if (c == nullptr || key == nullptr) return fail(MVSK_EINVAL, "null argument");
  Options& o = c->opt;
  const std::string k(key);
  auto pos = [&](double x) { return isfinite(x) && x > 0.0; };
  auto cnt = [&](double x, double lo, double hi) { return isfinite(x) && x == floor(x) && x >= lo && x <= hi; };
  if (k == "tau" && isfinite(v) && v >= 0.0 && v * c->n < 1.0) o.tau = v;
  else if (k == "eta" && pos(v)) o.eta = v;
  else if (k == "max_iter" && cnt(v, 1, 1000000)) o.max_iter = (int)v;
  else if (k == "pcg_max_iter" && cnt(v, 1, 1000000)) o.pcg_max_iter = (int)v;
  else if (k == "restart_iter" && cnt(v, 1, 1000000)) o.restart_iter1 = o.restart_iter2 = (int)v;
  else if (k == "restart_iter1" && cnt(v, 1, 1000000)) o.restart_iter1 = (int)v;
  else if (k == "restart_iter2" && cnt(v, 1, 1000000)) o.restart_iter2 = (int)v;
  else if (k == "restart_eta1" && pos(v)) o.restart_eta1 = v;
  else if (k == "restart_eta2" && pos(v)) o.restart_eta2 = v;
  else if (k == "max_elapsed" && v > 0.0) o.max_elapsed = v;
  else if (k == "krylov_tol" && pos(v)) o.krylov_tol = v;
  else if (k == "krylov_maxit" && cnt(v, 1, 10000)) o.krylov_maxit = (int)v;
  else if (k == "reg" && (isnan(v) || (isfinite(v) && v >= 0.0))) o.reg = v;
  else if (k == "probes" && cnt(v, 0, kMaxProbes)) o.probes = (int)v;
  else if (k == "probe_seed" && cnt(v, 0, 9007199254740992.0)) o.probe_seed = (unsigned long long)v;
  else if (k == "pref_scaling" && cnt(v, 0, 1)) o.pref_scaling = (int)v;
  else if (k == "release_ratio" && pos(v)) o.release_ratio = v;
  else if (k == "eps_act" && isfinite(v) && v >= 0.0) o.eps_act = v;
  else if (k == "oracle_prec" && cnt(v, 0, 2)) o.oracle_prec = (int)v;
  else if (k == "cal_rel_tol" && pos(v)) o.cal_rel_tol = v;
  else if (k == "stall_window" && cnt(v, 0, 15)) o.stall_window = (int)v;
  else if (k == "trace" && cnt(v, 0, 1)) o.trace = (int)v;
  else if (k == "graphs" && cnt(v, 0, 1)) c->use_graphs = v != 0.0;
  else if (k == "split_products" && cnt(v, 0, 1)) o.split_products = (int)v;
  else if (k == "batch_lanes" && cnt(v, 0, 1000000)) o.batch_lanes = (int)v;
  else if (k == "line_search" && cnt(v, 0, 1)) o.line_search = (int)v;
  else if (k == "group_calibration" && cnt(v, 0, 1)) o.group_cal = (int)v;
  else if (k == "face_products" && cnt(v, 0, 1)) o.face_products = (int)v;
  else if (k == "face_small" && cnt(v, 0, 2)) o.face_small = (int)v;
  else return fail(MVSK_EINVAL, "unknown option or bad value: %s = %g", key, v);
  if (c->prefs_set && k == "pref_scaling") mvsk_set_prefs(c, c->lam, c->target);
  return MVSK_OK;
}

mvsk_status mvsk_solve(mvsk_ctx* c, mvsk_config cfg, double tol, const double* w0, double* w_out, mvsk_info* info) {
  if (c == nullptr || w_out == nullptr) return fail(MVSK_EINVAL, "null argument");
  if (!c->prefs_set) return fail(MVSK_ESTATE, "mvsk_set_prefs must come first");
  if (!(tol > 0.0) || (cfg != MVSK_DIRECT && cfg != MVSK_PCG)) return fail(MVSK_EINVAL, "bad tol or configuration");
  double* w0d = nullptr;
  if (w0 != nullptr) {
    w0d = c->vec_scratch + 64;
    TRY(check_w0(c, w0, w0d));
  }
  const mvsk_status st = solve_with_target(c, cfg, tol, w0d, c->lam, c->target, info);
  if (st == MVSK_OK || st == MVSK_ENOTCONVERGED || st == MVSK_ETIMEOUT) {
    TRY(download_vec(c, w_out, c->in.x, c->n));
    TRY(sync(c));
  }
  return st;
}

mvsk_status mvsk_solve_batch(mvsk_ctx* c, mvsk_config cfg, int32_t B, const double* lambdas, const double* targets,
                             double tol, const double* W0, double* W_out, mvsk_info* infos) {
  if (c == nullptr || lambdas == nullptr || W_out == nullptr || B < 1) return fail(MVSK_EINVAL, "bad argument");
  std::vector<double> lam(4 * (size_t)B), tg((size_t)B, NAN);
  if (cudaMemcpy(lam.data(), lambdas, sizeof(double) * 4 * B, cudaMemcpyDefault) != cudaSuccess)
    return fail(MVSK_ECUDA, "copy of lambdas failed");
  if (targets != nullptr && cudaMemcpy(tg.data(), targets, sizeof(double) * B, cudaMemcpyDefault) != cudaSuccess)
    return fail(MVSK_ECUDA, "copy of targets failed");
  for (int b = 0; b < B; ++b)
    for (int q = 0; q < 4; ++q)
      if (!(lam[4 * (size_t)b + q] >= 0.0) || !isfinite(lam[4 * (size_t)b + q]))
        return fail(MVSK_EINVAL, "lambda[%d][%d] must be finite and >= 0", b, q);
  if (!(tol > 0.0)) return fail(MVSK_EINVAL, "bad tol");
  if (cfg == MVSK_PCG && c->dir_prec == P16 && c->opt.probes * 2 <= kTcCols && c->opt.probes + 1 <= kTcCols &&
      !c->opt.trace && c->use_graphs)
    return batch_solve(c, B, lam.data(), tg.data(), tol, W0, W_out, infos);
  mvsk_status first = MVSK_OK;
  for (int b = 0; b < B; ++b) {
    TRY(mvsk_set_prefs(c, &lam[4 * (size_t)b], tg[b]));
    const mvsk_status st = mvsk_solve(c, cfg, tol, W0 ? W0 + (size_t)b * c->n : nullptr, W_out + (size_t)b * c->n,
                                      infos ? infos + b : nullptr);
    if (st != MVSK_OK && st != MVSK_ENOTCONVERGED && st != MVSK_ETIMEOUT) return st;
    if (st != MVSK_OK && first == MVSK_OK) first = st;
  }
  return first;
}

mvsk_status mvsk_eval(mvsk_ctx* c, const double* w, double* f, double* grad, double* kkt) {
  if (c == nullptr || w == nullptr) return fail(MVSK_EINVAL, "null argument");
  if (!c->prefs_set) return fail(MVSK_ESTATE, "mvsk_set_prefs must come first");
  TRY(init_state(c, MVSK_PCG, 1.0, c->c));
  TRY(upload_vec(c, c->in.x, w, c->n));
  double ev[3];
  TRY(eval_here(c, ev));
  if (f) *f = ev[0];
  if (kkt) *kkt = ev[1];
  if (grad) {
    TRY(download_vec(c, grad, c->in.g, c->n));
    TRY(sync(c));
  }
  return MVSK_OK;
}

mvsk_status mvsk_oracle_hvp(mvsk_ctx* c, const double* w, const double* v, double* out) {
  if (c == nullptr || w == nullptr || v == nullptr || out == nullptr) return fail(MVSK_EINVAL, "null argument");
  if (!c->prefs_set) return fail(MVSK_ESTATE, "mvsk_set_prefs must come first");
  Inst& s = c->in;
  TRY(upload_vec(c, s.x, w, c->n));
  TRY(upload_vec(c, s.d, v, c->n));
  TRY(pass_fwd_z(c, s.x, s.z));
  PassArgs a = pass_args(c);
  a.in[0] = s.d;
  a.z = s.z;
  TRY(run_pass(c, c->opt.oracle_prec, M_HVP, 1, a));
  TRY(reduce_cols(c, c->opt.oracle_prec, 1, s.at, c->ld, nullptr, 0.0, nullptr, nullptr));
  TRY(download_vec(c, out, s.at, c->n));
  return sync(c);
}

mvsk_status mvsk_oracle_third(mvsk_ctx* c, const double* w, const double* u, const double* v, double* out) {
  if (c == nullptr || w == nullptr || u == nullptr || v == nullptr || out == nullptr)
    return fail(MVSK_EINVAL, "null argument");
  if (!c->prefs_set) return fail(MVSK_ESTATE, "mvsk_set_prefs must come first");
  Inst& s = c->in;
  TRY(upload_vec(c, s.x, w, c->n));
  TRY(upload_vec(c, s.d, u, c->n));
  TRY(upload_vec(c, s.dstep, v, c->n));
  TRY(pass_fwd_z(c, s.x, s.z));
  PassArgs a = pass_args(c);
  a.in[0] = s.d;
  a.in[1] = s.dstep;
  a.z = s.z;
  TRY(run_pass(c, c->opt.oracle_prec, M_THIRD, 2, a));
  TRY(reduce_cols(c, c->opt.oracle_prec, 1, s.at, c->ld, nullptr, 0.0, nullptr, nullptr));
  TRY(download_vec(c, out, s.at, c->n));
  return sync(c);
}

mvsk_status mvsk_oracle_gram(mvsk_ctx* c, const double* w, double* G) {
  if (c == nullptr || w == nullptr || G == nullptr) return fail(MVSK_EINVAL, "null argument");
  if (!c->prefs_set) return fail(MVSK_ESTATE, "mvsk_set_prefs must come first");
  Inst& s = c->in;
  TRY(upload_vec(c, s.x, w, c->n));
  TRY(pass_fwd_z(c, s.x, s.z));
  TRY(gram_into(c, s.z, c->opt.oracle_prec == 1 ? P16 : P64));
  CU(cudaMemcpy2DAsync(G, sizeof(double) * c->n, c->Gm, sizeof(double) * c->ld, sizeof(double) * c->n, c->n,
                       cudaMemcpyDefault, c->stream));
  return sync(c);
}

// out_b = A V_b (transpose = 0, T values) or A^T V_b (transpose = 1,
// n values) with the emulated-FP64 tensor-core product; device pointers.
mvsk_status mvsk_product(mvsk_ctx* c, int32_t transpose, int32_t nvec, const double* V, int64_t ldv, double* out,
                         int64_t ldo) {
  if (c == nullptr || V == nullptr || out == nullptr) return fail(MVSK_EINVAL, "null argument");
  if (nvec < 1 || nvec > kOzMaxB) return fail(MVSK_EINVAL, "nvec must be in [1, %d]", kOzMaxB);
  const long long K = transpose ? c->T : c->n, M = transpose ? c->n : c->T;
  if (ldv < K || ldo < M) return fail(MVSK_EINVAL, "leading dimension too small");
  cudaPointerAttributes pa, pb;
  CU(cudaPointerGetAttributes(&pa, V));
  CU(cudaPointerGetAttributes(&pb, out));
  if (pa.type != cudaMemoryTypeDevice || pb.type != cudaMemoryTypeDevice)
    return fail(MVSK_EINVAL, "mvsk_product takes device pointers");
  const int Bp = oz_bp(nvec);
  int splits = 0;
  TRY(oz_product(c, transpose ? 1 : 0, V, ldv, nvec, Bp, nullptr, &splits));
  const OzBuf& o = c->oz;
  const long long Mp = transpose ? o.MpB : o.MpF;
  k_oz_store<<<dim3((unsigned)((M + 255) / 256), (unsigned)nvec), 256, 0, c->stream>>>(
      o.part, splits, Bp, Mp, M, nvec, transpose ? o.eB : o.eF, transpose ? o.fB : o.fF, 1.0, out, ldo);
  c->launches += 1;
  CU(cudaGetLastError());
  return sync(c);
}

mvsk_status mvsk_batch_hvp(mvsk_ctx* c, int32_t B, const double* C, const double* X, const double* nuhat,
                           const double* maskF, int32_t nc, const double* V, double* HV, double* Gnu, double* diagG,
                           int32_t path[2]) {
  if (c == nullptr || C == nullptr || X == nullptr || nuhat == nullptr || V == nullptr || HV == nullptr ||
      Gnu == nullptr || diagG == nullptr)
    return fail(MVSK_EINVAL, "null argument");
  return batch_hvp_export(c, B, C, X, nuhat, maskF, nc, V, HV, Gnu, diagG, path);
}

mvsk_status mvsk_batch_third(mvsk_ctx* c, int32_t B, const double* C, const double* X, const double* maskF,
                             int32_t K, const double* U, const double* P, double* at) {
  if (c == nullptr || C == nullptr || X == nullptr || U == nullptr || P == nullptr || at == nullptr)
    return fail(MVSK_EINVAL, "null argument");
  return batch_third_export(c, B, C, X, maskF, K, U, P, at);
}

mvsk_status mvsk_oracle_ls(mvsk_ctx* c, const double* w, const double* d, double coef[5], double* alpha_max) {
  if (c == nullptr || w == nullptr || d == nullptr || coef == nullptr) return fail(MVSK_EINVAL, "null argument");
  if (!c->prefs_set) return fail(MVSK_ESTATE, "mvsk_set_prefs must come first");
  Inst& s = c->in;
  TRY(init_state(c, MVSK_PCG, 1.0, c->c));
  TRY(upload_vec(c, s.x, w, c->n));
  TRY(upload_vec(c, s.d, d, c->n));
  TRY(pass_fwd_z(c, s.x, s.z));
  TRY(pass_ls(c, s.d, nullptr));
  double* dc = c->vec_scratch + 32;
  k_ls_coef_only<<<1, kVT, 0, c->stream>>>(s, c->spart, c->grid, s.d, dc);
  k_alpha_max<<<1, kVT, 0, c->stream>>>(s.x, s.d, c->n, c->opt.tau, dc + 5);
  CU(cudaGetLastError());
  double h[6];
  CU(cudaMemcpyAsync(h, dc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  TRY(sync(c));
  for (int q = 0; q < 5; ++q) coef[q] = h[q];
  if (alpha_max) *alpha_max = h[5];
  return MVSK_OK;
}

mvsk_status mvsk_oracle_direction(mvsk_ctx* c, mvsk_config cfg, const double* w, int32_t iteration, double* d_out) {
  if (c == nullptr || w == nullptr || d_out == nullptr) return fail(MVSK_EINVAL, "null argument");
  if (!c->prefs_set) return fail(MVSK_ESTATE, "mvsk_set_prefs must come first");
  Inst& s = c->in;
  TRY(init_state(c, cfg, 1.0, c->c));
  int h2[2] = {1, iteration};
  CU(cudaMemcpyAsync(c->si + SI_DIRONLY, &h2[0], sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->si + SI_ITER, &h2[1], sizeof(int), cudaMemcpyHostToDevice, c->stream));
  TRY(upload_vec(c, s.x, w, c->n));
  TRY(pass_valgrad(c, s.x, s.z, s.g, nullptr));
  k_face<<<1, kVT, 0, c->stream>>>(s, c->spart, c->grid);
  CU(cudaGetLastError());
  c->launches += 5;  // k_face, k_decide1, k_decide2, k_end_iter (+1 below)
  TRY(direction(c, cfg));
  TRY(download_vec(c, d_out, s.d, c->n));
  return sync(c);
}

mvsk_status mvsk_project_slice(mvsk_ctx* c, const double* v, double tau, double* out) {
  if (c == nullptr || v == nullptr || out == nullptr) return fail(MVSK_EINVAL, "null argument");
  if (!(tau >= 0.0) || !(tau * c->n < 1.0)) return fail(MVSK_EINVAL, "tau out of range");
  Inst& s = c->in;
  TRY(upload_vec(c, s.d, v, c->n));
  k_project<<<1, kVT, 0, c->stream>>>(s.d, c->n, tau, s.dstep);
  CU(cudaGetLastError());
  TRY(download_vec(c, out, s.dstep, c->n));
  return sync(c);
}

mvsk_status mvsk_column_stats(mvsk_ctx* c, double* mu, double* sigma) {
  if (c == nullptr || mu == nullptr || sigma == nullptr) return fail(MVSK_EINVAL, "null argument");
  Inst& s = c->in;
  k_colstd<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->A64, c->T, c->n, c->ld, s.dstep);
  CU(cudaGetLastError());
  TRY(download_vec(c, mu, c->mu, c->n));
  TRY(download_vec(c, sigma, s.dstep, c->n));
  return sync(c);
}

mvsk_status mvsk_quartic_argmin(mvsk_ctx* c, const double coef[5], double amax, double* alpha) {
  if (c == nullptr || coef == nullptr || alpha == nullptr) return fail(MVSK_EINVAL, "null argument");
  double* dc = c->vec_scratch + 40;
  CU(cudaMemcpyAsync(dc, coef, 5 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  k_quartic<<<1, 32, 0, c->stream>>>(dc, amax, dc + 5);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(alpha, dc + 5, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return sync(c);
}

// Label of profiler kind `kind` (see kKernelNames and prof_begin).
static void kind_name(int kind, char* out, size_t len) {
  static const char* modes[] = {"valgrad", "fwd", "hvp", "hvpdiag", "third", "rhat", "back", "ls"};
  static const char* precs[] = {"fp64", "bf16", "fp32"};
  if (kind < 400)
    snprintf(out, len, "rowpass_%s_%s_%d", precs[(kind / 128) % 3], modes[(kind / 8) % 16 % 8], kind % 8);
  else if (kind < 680)
    snprintf(out, len, "gemm_tc_bf16_n%d", kind - 400);
  else if (kind >= 680 && kind <= 683)
    snprintf(out, len, "oz_gemm_%s%s", (kind & 1) ? "bwd" : "fwd", kind >= 682 ? "_gated" : "");
  else if (kind == 684 || kind == 685)
    snprintf(out, len, "oz_gemm_fwd_u%s", kind == 685 ? "_gated" : "");
  else if (kind >= kKindNamed && kind < kKindNamed + NK_COUNT)
    snprintf(out, len, "%s", kKernelNames[kind - kKindNamed]);
  else
    snprintf(out, len, "kernel_%d", kind);
}

mvsk_status mvsk_profile_only(mvsk_ctx* c, const char* prefix) {
  if (c == nullptr) return fail(MVSK_EINVAL, "null context");
  c->prof_sel.clear();
  if (prefix == nullptr) return MVSK_OK;
  c->prof_sel.assign(kProfKinds, 0);
  // a comma-separated list of prefixes selects the union of their kinds
  const std::string all(prefix);
  size_t p0 = 0;
  char nm[64];
  while (p0 <= all.size()) {
    size_t p1 = all.find(',', p0);
    if (p1 == std::string::npos) p1 = all.size();
    const std::string pre = all.substr(p0, p1 - p0);
    for (int k = 0; k < kProfKinds; ++k) {
      kind_name(k, nm, sizeof(nm));
      if (strncmp(nm, pre.c_str(), pre.size()) == 0) c->prof_sel[k] = 1;
    }
    p0 = p1 + 1;
  }
  return MVSK_OK;
}

mvsk_status mvsk_profile_stride(mvsk_ctx* c, int32_t k) {
  if (c == nullptr) return fail(MVSK_EINVAL, "null context");
  if (k < 1) return fail(MVSK_EINVAL, "profile stride must be >= 1 (got %d)", (int)k);
  c->prof_stride = k;
  c->prof_count.clear();
  return MVSK_OK;
}

mvsk_status mvsk_profile_enable(mvsk_ctx* c, int32_t on) {
  if (c == nullptr) return fail(MVSK_EINVAL, "null context");
  CU(cudaStreamSynchronize(c->stream));
  c->prof_on = on != 0;
  if (on) {
    c->prof_count.clear();
    c->ev_used = 0;
    c->ev_kind.clear();
    c->ev_work.clear();
    c->ev_uscale.clear();
    c->ev_in_graph.clear();
    c->launches = 0;
    c->prof_n.assign(kProfKinds, 0);
    c->prof_ms.assign(kProfKinds, 0.0);
    c->prof_work.assign(kProfKinds, 0.0);
    c->ev_graph_begin = c->ev_graph_end = 0;
  }
  return MVSK_OK;
}

mvsk_status mvsk_profile_read(mvsk_ctx* c, mvsk_prof_entry* out, int32_t max, int32_t* count, int64_t* kernel_launches) {
  if (c == nullptr) return fail(MVSK_EINVAL, "null context");
  CU(cudaStreamSynchronize(c->stream));
  if (c->prof_n.empty()) {
    if (count) *count = 0;
    if (kernel_launches) *kernel_launches = c->launches;
    return MVSK_OK;
  }
  // pairs recorded by direct launches (graph pairs were folded in after each replay)
  std::vector<long long> n = c->prof_n;
  std::vector<double> ms = c->prof_ms;
  std::vector<double> wk = c->prof_work;
  for (size_t q = 0; q < c->ev_kind.size(); ++q) {
    if (c->ev_in_graph[q]) continue;
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, c->ev_pool[2 * q], c->ev_pool[2 * q + 1]));
    n[c->ev_kind[q]] += 1;
    ms[c->ev_kind[q]] += t;
    wk[c->ev_kind[q]] += c->ev_work[q];
  }
    int k = 0;
  for (int kind = 0; kind < kProfKinds; ++kind) {
    if (n[kind] == 0) continue;
    if (k < max) {
      kind_name(kind, out[k].name, sizeof(out[k].name));
      out[k].launches = n[kind];
      out[k].total_ms = ms[kind];
      out[k].bytes_per_launch = wk[kind] / (double)n[kind];
    }
    ++k;
  }
  if (count) *count = k;
  if (kernel_launches) *kernel_launches = c->launches;
  return MVSK_OK;
}

const char* mvsk_last_error(const mvsk_ctx*) { return g_err; }

void mvsk_destroy(mvsk_ctx* c) {
  if (c == nullptr) return;
  cudaDeviceSynchronize();
  for (void* p : c->allocs) cudaFree(p);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (void* p : c->batch.mem) cudaFree(p);
  if (c->batch.Gq != nullptr) cudaFree(c->batch.Gq);
  if (c->batch.Wq != nullptr) cudaFree(c->batch.Wq);
  if (c->batch.Zq != nullptr) cudaFree(c->batch.Zq);
  if (c->batch.gpool != nullptr) cudaFree(c->batch.gpool);
  if (c->batch.si_h != nullptr) cudaFreeHost(c->batch.si_h);
  if (c->batch.ev_h != nullptr) cudaFreeHost(c->batch.ev_h);
  if (c->batch.sd_h != nullptr) cudaFreeHost(c->batch.sd_h);
  if (c->batch.q_si != nullptr) cudaFreeHost(c->batch.q_si);
  if (c->batch.q_ev != nullptr) cudaFreeHost(c->batch.q_ev);
  if (c->hword != nullptr) cudaFreeHost(c->hword);
  if (c->own_stream != nullptr) cudaStreamDestroy(c->own_stream);
  delete c;
}

}  // extern "C"

namespace mvsk {

void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

size_t rowpass_smem(int prec, int mode, int nin, int ld, int* stages) {
  if (prec == P64) return rowpass_smem_f64(mode, nin, ld, stages);
  if (prec == P16) return rowpass_smem_bf16(mode, nin, ld, stages);
  return rowpass_smem_f32(mode, nin, ld, stages);
}

cudaError_t rowpass_launch(int prec, int mode, int nin, const PassArgs& a, int grid, size_t smem, cudaStream_t st) {
  if (prec == P64) return rowpass_launch_f64(mode, nin, a, grid, smem, st);
  if (prec == P16) return rowpass_launch_bf16(mode, nin, a, grid, smem, st);
  return rowpass_launch_f32(mode, nin, a, grid, smem, st);
}

}  // namespace mvsk
