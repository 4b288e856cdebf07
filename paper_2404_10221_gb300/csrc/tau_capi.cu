// C ABI of the τ-preconditioned GMRES solver: problem lifetime, one-time setup, the
// Crank–Nicolson step as a CUDA graph with device-side GMRES loop control, and the
// operator-level entry points.  See include/tau_rsfde.h for the contract of every call.
#include "tau_rsfde.h"
#include "tau_internal.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include <sys/stat.h>

using namespace tau;

namespace {

thread_local std::string g_err;
// kernels enqueued by this thread (used to count the kernels of the step graph)
thread_local int64_t tl_launches = 0;

tau_status fail(tau_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t _e = (call);                                                                 \
    if (_e != cudaSuccess) return fail(TAU_ECUDA, "%s: %s", #call, cudaGetErrorString(_e));  \
  } while (0)

#define KL(call)          \
  do {                    \
    ++tl_launches;        \
    CK(call);             \
  } while (0)

#define TRY(call)                       \
  do {                                  \
    tau_status _s = (call);             \
    if (_s != TAU_OK) return _s;        \
  } while (0)

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

void tau::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

struct tau_problem {
  tau_problem_desc desc{};
  cudaStream_t st = nullptr;    // caller's stream: every operation is enqueued here
  cudaStream_t cap = nullptr;   // library stream used only to record the step graph
  int d = 0;
  int n[3] = {1, 1, 1};
  int64_t n_tot = 0;
  double dt = 0, h[3] = {0, 0, 0}, eta[3] = {0, 0, 0};
  int route[3] = {0, 0, 0};
  // device buffers
  double *V = nullptr, *u = nullptr, *b = nullptr, *A = nullptr, *C = nullptr, *E = nullptr, *Fdt = nullptr,
         *invmu = nullptr, *tmp = nullptr;
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *gv = nullptr, *h1 = nullptr, *h2 = nullptr, *y = nullptr;
  double *pdots = nullptr, *pnorm = nullptr, *escan = nullptr;
  GmresDev* g = nullptr;
  int* iters = nullptr;
  double2* spec[3] = {nullptr, nullptr, nullptr};
  // CHIRP route: Toeplitz transform length KT (power of two >= n+1), DST convolution length MC
  // (power of two >= 2n; Bluestein DFT of length n+1 for two lines at once), the chirp c_m, the
  // kernel spectrum and the length-MC twiddles
  int KT[3] = {0, 0, 0}, MC[3] = {0, 0, 0};
  double2 *chirp[3] = {nullptr, nullptr, nullptr}, *bhat[3] = {nullptr, nullptr, nullptr},
          *twM[3] = {nullptr, nullptr, nullptr};
  float2 *chirp32[3] = {nullptr, nullptr, nullptr}, *bhat32[3] = {nullptr, nullptr, nullptr},
         *twM32[3] = {nullptr, nullptr, nullptr};
  df64x2 *chirp_df[3] = {nullptr, nullptr, nullptr}, *bhat_df[3] = {nullptr, nullptr, nullptr},
         *twM_df[3] = {nullptr, nullptr, nullptr};
  double2 *twK[3] = {nullptr, nullptr, nullptr}, *twK2[3] = {nullptr, nullptr, nullptr};
  // LONG route (d = 1): four-step FFT tables per element type (work and ybuf shared by all three)
  LongTab<double> lt64[3] = {};
  LongTab<float> lt32[3] = {};
  LongTab<df64> ltdf[3] = {};
  // mixed form: tensor-core DST-I mode products of the FP32 τ solve (dimensions with n <= 256)
  TcTab tc[3] = {};
  bool tc_on[3] = {false, false, false};
  int* tc_err = nullptr;
  // mixed form: split-TF32 tensor-core Toeplitz matvec (every dimension n <= 256) and the second
  // pair of FP32 channel buffers its passes alternate with
  bool tcm = false;
  float *A2 = nullptr, *C2 = nullptr;
  // device flag: tmp holds the FP64 residual of the current solution (end of a mixed step), so the
  // next right-hand side can be formed from it (tau_mixed.cu)
  int* rres = nullptr;
  double *s[3] = {nullptr, nullptr, nullptr}, *sintab[3] = {nullptr, nullptr, nullptr};
  double *beta[3] = {nullptr, nullptr, nullptr}, *q[3] = {nullptr, nullptr, nullptr};
  double *e_tc = nullptr, *f_tc = nullptr, *psi_tc = nullptr;
  // fields given as caller-owned device arrays (tau_set_fields_device)
  const double *e_dev = nullptr, *f_dev = nullptr, *psi_dev = nullptr;
  int64_t e_step = 0, f_step = 0;
  double *e_sp[3] = {nullptr, nullptr, nullptr}, *f_hsp[3] = {nullptr, nullptr, nullptr},
         *psi_sp[3] = {nullptr, nullptr, nullptr};
  int re = 0, rf = 0, rp = 0;
  bool fields_set = false, setup_done = false;
  double ebar = 0, ehat = 0, echeck = 0;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;
  int64_t k_pro = 0, k_body = 0, k_epi = 0;  // kernels per prologue / GMRES iteration / epilogue
  // mixed precision (FP64 refinement around an FP32 flexible GMRES)
  bool mixed = false;
  int kin = 0;                                 // inner iteration cap
  double *X = nullptr;                         // FP64 iterate of the refinement
  float *V32 = nullptr, *Z32 = nullptr, *A32 = nullptr, *C32 = nullptr, *invmu32 = nullptr, *E32 = nullptr;
  double *Hin = nullptr, *csin = nullptr, *snin = nullptr, *gvin = nullptr, *h1in = nullptr, *h2in = nullptr,
         *yin = nullptr;
  GmresDev* gin = nullptr;
  IRDev* ir = nullptr;
  int* sweeps = nullptr;
  float2 *spec32[3] = {nullptr, nullptr, nullptr}, *twK32[3] = {nullptr, nullptr, nullptr},
         *twK2_32[3] = {nullptr, nullptr, nullptr};
  float *s32[3] = {nullptr, nullptr, nullptr}, *sintab32[3] = {nullptr, nullptr, nullptr};
  int64_t k_ir_pre = 0, k_ir_post = 0;         // kernels of one refinement sweep around the inner loop
  // autotuning of this problem's setup: measure new choices, and/or take recorded ones
  bool tune_measure = false, tune_records = false;
  int route_src[3] = {0, 0, 0};                 // 0 rule or forced, 1 measured, 2 recorded measurement
  double route_ms[3] = {0, 0, 0}, route_alt_ms[3] = {0, 0, 0};
  // the autotuner's tile per element type and dimension: lines per CTA, plus 1 << 16 when the CTA
  // has 256 threads (the wide line-pass variant); 0: the shared-memory heuristic, 128 threads
  int lpb_tuned[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                                                          // (FP64, FP32, double-float)
  // double-float precision (TAU_DF64): solver vectors live in the FP64 buffers above as df64 pairs
  bool dfm = false;
  df64 *Edf = nullptr, *Fdf = nullptr, *invmu_df = nullptr;
  // mixed form: the outer residual b - A x as double-float line passes (X and tmp then hold df64
  // pairs, b is copied to bdf), chosen at setup where its rounding floor is below refine_tol
  bool res_df = false;
  df64* bdf = nullptr;
  // grouped batch: the group's loop-condition aggregators ([0] refinement control, [1] Givens);
  // set while the batch graph is recorded (use_cond 2), NULL otherwise
  GroupCtl* gctl = nullptr;
  // two-sided method (TAU_TPGM): sine-basis diagonals of P^{-1/2} and P^{-1/2} B^{-1}
  int tpgm = 0;
  double *pmh = nullptr, *pmhb = nullptr;
  // Strang circulant comparison method (TAU_SPGM): Fourier-basis diagonal 1/p_c, sine-basis 1/beta,
  // and per dimension the Hartley table and the DFT eigenvalues of s(B_i), s(S_i)
  int spgm = 0;
  double *pcinv = nullptr, *binv = nullptr;
  double *cas[3] = {nullptr, nullptr, nullptr}, *sb[3] = {nullptr, nullptr, nullptr},
         *ss[3] = {nullptr, nullptr, nullptr};
  df64x2 *spec_df[3] = {nullptr, nullptr, nullptr}, *twK_df[3] = {nullptr, nullptr, nullptr},
         *twK2_df[3] = {nullptr, nullptr, nullptr};
  df64 *s_df[3] = {nullptr, nullptr, nullptr}, *sintab_df[3] = {nullptr, nullptr, nullptr};
  int64_t fields_m = -1;                      // step whose e and dt*F sit in E / Fdt
  int* h_done = nullptr;  // pinned flag for the host-loop fallback
  std::vector<void*> allocs;
  int64_t bytes = 0;
  int64_t m_host = 0;
};

namespace {

tau_status dalloc(tau_problem* p, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TAU_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  p->allocs.push_back(*ptr);
  p->bytes += (int64_t)bytes;
  return TAU_OK;
}

template <typename T>
tau_status dalloc_n(tau_problem* p, T** ptr, size_t count) {
  return dalloc(p, reinterpret_cast<void**>(ptr), count * sizeof(T));
}

template <typename T>
tau_status upload(tau_problem* p, T** dst, const T* src, size_t count) {
  TRY(dalloc_n(p, dst, count));
  CK(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
  return TAU_OK;
}

FieldDev field_dev(const tau_problem* p) {
  FieldDev f{};
  f.d = p->d;
  for (int i = 0; i < 3; ++i) {
    f.n[i] = i < p->d ? p->n[i] : 1;
    f.e_sp[i] = p->e_sp[i];
    f.f_hsp[i] = p->f_hsp[i];
  }
  f.n_tot = p->n_tot;
  f.re = p->re;
  f.rf = p->rf;
  f.e_tc = p->e_tc;
  f.f_tc = p->f_tc;
  f.dt = p->dt;
  f.e_dev = p->e_dev;
  f.e_step = p->e_step;
  f.f_dev = p->f_dev;
  f.f_step = p->f_step;
  for (int i = 0; i < 3; ++i) {
    const double a = i < p->d ? p->desc.alpha[i] : 0.0;
    f.hw[i][0] = a / 24.0;
    f.hw[i][1] = 1.0 - a / 12.0;
  }
  return f;
}

// host-side conversion of a scalar to the element type (double-float: hi = fl(v), lo = fl(v - hi))
template <typename T> T host_cast(double v) { return (T)v; }
template <> df64 host_cast<df64>(double v) {
  const float h = (float)v;
  return df64{h, (float)(v - (double)h)};
}

template <typename T> constexpr int prec_index() {
  return std::is_same<T, double>::value ? 0 : (std::is_same<T, float>::value ? 1 : 2);
}

template <typename T>
void set_lpb(PassT<T>& P, int lpb) {
  // the line-pass kernel maps threads to lines with shifts: a power of two
  if (lpb < 1) lpb = 1;
  while (lpb & (lpb - 1)) lpb &= lpb - 1;
  P.lpb = lpb;
  const int64_t outer = P.nlines / P.inner;
  P.ntiles = P.ax == 0 ? (P.nlines + lpb - 1) / lpb : outer * ((P.inner + lpb - 1) / lpb);
}

template <typename T>
PassT<T> base_pass_t(const tau_problem* p, int ax) {
  PassT<T> P{};
  P.ax = ax;
  P.len = p->n[ax];
  int64_t inner = 1;
  for (int i = 0; i < ax; ++i) inner *= p->n[i];
  P.inner = inner;
  P.nlines = p->n_tot / P.len;
  DimDataT<T>& D = P.dim;
  D.n = p->n[ax];
  D.K = p->n[ax] + 1;
  D.route = p->route[ax];
  D.bdiag = host_cast<T>(1.0 - p->desc.alpha[ax] / 12.0);
  D.boff = host_cast<T>(p->desc.alpha[ax] / 24.0);
  D.dsc = host_cast<T>(std::sqrt(2.0 / (double)(p->n[ax] + 1)));
  D.eta = p->eta[ax];
  if constexpr (std::is_same<T, double>::value) {
    D.spec = p->spec[ax];
    D.s = p->s[ax];
    D.sintab = p->sintab[ax];
    D.twK = p->twK[ax];
    D.twK2 = p->twK2[ax];
    D.cas = p->cas[ax];
    D.chirp = p->chirp[ax];
    D.bhat = p->bhat[ax];
    D.twM = p->twM[ax];
    P.in_base = P.out_base = p->V;
  } else if constexpr (std::is_same<T, df64>::value) {
    D.spec = p->spec_df[ax];
    D.s = p->s_df[ax];
    D.sintab = p->sintab_df[ax];
    D.twK = p->twK_df[ax];
    D.twK2 = p->twK2_df[ax];
    D.chirp = p->chirp_df[ax];
    D.bhat = p->bhat_df[ax];
    D.twM = p->twM_df[ax];
    P.in_base = P.out_base = reinterpret_cast<df64*>(p->V);
  } else {
    D.spec = p->spec32[ax];
    D.s = p->s32[ax];
    D.sintab = p->sintab32[ax];
    D.twK = p->twK32[ax];
    D.twK2 = p->twK2_32[ax];
    D.chirp = p->chirp32[ax];
    D.bhat = p->bhat32[ax];
    D.twM = p->twM32[ax];
  }
  if (D.route == ROUTE_CHIRP) {
    D.K = p->KT[ax];
    D.M = p->MC[ax];
  }
  if constexpr (std::is_same<T, double>::value) D.lng = &p->lt64[ax];
  else if constexpr (std::is_same<T, df64>::value) D.lng = &p->ltdf[ax];
  else D.lng = &p->lt32[ax];
  // shared memory per line: the line (N reals) plus the transform line (2K reals, FFT route) or a
  // second copy (N, dense route).  24 KB of lines per CTA lets 8 CTAs of 128 threads share an SM.
  size_t rs = 2 * (size_t)P.len;   // dense route: the line and its outputs
  if (D.route == ROUTE_FFT || D.route == ROUTE_CHIRP) rs = 2 * (size_t)D.K;
  const size_t per_line = sizeof(T) * ((size_t)P.len + rs);
  int64_t lpb = (int64_t)(24576 / per_line);
  if (lpb < 1) lpb = 1;
  // chirp route: two lines share one DST convolution; a single line pays for a pair's buffer anyway
  if (D.route == ROUTE_CHIRP && lpb < 2) lpb = 2;
  if (lpb > 16) lpb = 16;
  const int64_t cap = ax == 0 ? P.nlines : inner;
  const int tuned = p->lpb_tuned[prec_index<T>()][ax];
  if (tuned > 0) {
    lpb = tuned & 0xFFFF;
    P.tpb = (tuned >> 16) ? 256 : 128;
  }
  if (lpb > cap) lpb = cap;
  set_lpb(P, (int)lpb);
  P.vstride = p->n_tot;
  return P;
}

Pass base_pass(const tau_problem* p, int ax) { return base_pass_t<double>(p, ax); }

// I/O of a pass chain: plain pointers, or vectors selected on the device by the Arnoldi index j
// (sel 1: base + j * n_tot, sel 2: base + (j+1) * n_tot).
template <typename T>
struct ChainT {
  const T* x = nullptr;
  T* out = nullptr;
  int in_sel = 0, out_sel = 0;
  T* in_base = nullptr;
  T* out_base = nullptr;
  const GmresDev* g = nullptr;
  const T* diag = nullptr;   // sine-basis diagonal of the DST-diag-DST tail (default 1/mu)
};
using ChainIO = ChainT<double>;

template <typename T>
tau_status enq(const PassT<T>& P, cudaStream_t st) {
  if (P.dim.route == ROUTE_LONG) {
    tl_launches += long_launches(P) - 1;
    KL(launch_long(P, *P.dim.lng, st));
    return TAU_OK;
  }
  KL(launch_pass(P, st));
  return TAU_OK;
}

template <typename T> const T* invmu_of(const tau_problem* p);
template <> const double* invmu_of<double>(const tau_problem* p) { return p->invmu; }
template <> const float* invmu_of<float>(const tau_problem* p) { return p->invmu32; }
template <> const df64* invmu_of<df64>(const tau_problem* p) { return p->invmu_df; }
template <typename T> T* chanA(const tau_problem* p);
template <typename T> T* chanC(const tau_problem* p);
template <> double* chanA<double>(const tau_problem* p) { return p->A; }
template <> double* chanC<double>(const tau_problem* p) { return p->C; }
template <> float* chanA<float>(const tau_problem* p) { return p->A32; }
template <> float* chanC<float>(const tau_problem* p) { return p->C32; }
template <> df64* chanA<df64>(const tau_problem* p) { return reinterpret_cast<df64*>(p->A); }
template <> df64* chanC<df64>(const tau_problem* p) { return reinterpret_cast<df64*>(p->C); }
// coefficient e of the current step in the pass element type
template <typename T> const T* e_of(const tau_problem* p);
template <> const double* e_of<double>(const tau_problem* p) { return p->E; }
template <> const df64* e_of<df64>(const tau_problem* p) { return p->Edf; }
template <> const float* e_of<float>(const tau_problem* p) { return p->E32; }

template <typename T>
void wire_in(PassT<T>& P, const ChainT<T>& io, bool from_x) {
  if (from_x) {
    P.in_a = io.x;
    P.in_sel = io.in_sel;
    if (io.in_base) P.in_base = io.in_base;
  } else {
    P.in_a = io.out;
    P.in_sel = io.out_sel;
    if (io.out_base) P.in_base = io.out_base;
  }
}

template <typename T>
void wire_out(PassT<T>& P, const ChainT<T>& io) {
  P.out_a = io.out;
  P.out_sel = io.out_sel;
  if (io.out_base) P.out_base = io.out_base;
}

// DST along dims top..1 (descending), DST·(1/mu)·DST along dim 0, DST along dims 1..d-1,
// reading `x` in the first pass and working in place on `out` afterwards.
template <typename T>
tau_status enq_minv_tail(tau_problem* p, cudaStream_t st, const ChainT<T>& io, int top, bool first_reads_x) {
  bool rd = first_reads_x;
  auto dst_pass = [&](int ax, int post) -> tau_status {
    PassT<T> P = base_pass_t<T>(p, ax);
    P.post = post;
    P.invmu = io.diag ? io.diag : invmu_of<T>(p);
    P.g = io.g;
    wire_in(P, io, rd);
    wire_out(P, io);
    rd = false;
    if constexpr (std::is_same<T, float>::value) {
      if (p->tc_on[ax]) {   // tensor-core mode products (DST, or DST·(1/mu)·DST as two of them)
        const bool mu = post == POST_DST_MU_DST;
        KL(launch_tc_dst(P, p->tc[ax], mu ? P.invmu : nullptr, false, st));
        if (mu) KL(launch_tc_dst(P, p->tc[ax], nullptr, true, st));
        return TAU_OK;
      }
    }
    return enq(P, st);
  };
  for (int ax = top; ax >= 1; --ax) TRY(dst_pass(ax, POST_DST));
  TRY(dst_pass(0, POST_DST_MU_DST));
  for (int ax = 1; ax < p->d; ++ax) TRY(dst_pass(ax, POST_DST));
  return TAU_OK;
}

// out = finish( B(e∘x) + sgn*sum_i eta_i (..S_i..) x ), optionally followed by M^{-1}.
template <typename T>
tau_status enq_mv(tau_problem* p, cudaStream_t st, const ChainT<T>& io, double sgn, int finish, const T* src,
                  bool precond, const int* skip = nullptr) {
  const int d = p->d;
  if constexpr (std::is_same<T, float>::value) {
    if (p->tcm && finish == FIN_NONE && !precond) {
      // split-TF32 tensor-core passes; the channels alternate between (A32, C32) and (A2, C2)
      float* ba[2] = {p->A32, p->A2};
      float* bc[2] = {p->C32, p->C2};
      for (int ax = 0; ax < d; ++ax) {
        PassT<float> P = base_pass_t<float>(p, ax);
        P.skip = skip;
        P.seta = sgn * p->eta[ax];
        P.g = io.g;
        P.e = e_of<float>(p);
        const bool first = ax == 0, last = ax == d - 1;
        const float* c_in = first ? io.x : bc[(ax - 1) & 1];
        float* c_base = first ? io.in_base : nullptr;
        const int c_sel = first ? io.in_sel : 0;
        const float* a_in = first ? nullptr : ba[(ax - 1) & 1];
        float* out_a = last ? io.out : ba[ax & 1];
        float* out_base = last ? io.out_base : nullptr;
        const int out_sel = last ? io.out_sel : 0;
        float* out_c = last ? nullptr : bc[ax & 1];
        KL(launch_tc_mv(P, p->tc[ax], c_in, c_base, c_sel, a_in, out_a, out_base, out_sel, out_c, first, last, st));
      }
      return TAU_OK;
    }
  }
  for (int ax = 0; ax < d; ++ax) {
    PassT<T> P = base_pass_t<T>(p, ax);
    P.skip = skip;
    P.mv = 1;
    P.first = ax == 0;
    P.last = ax == d - 1;
    P.seta = sgn * p->eta[ax];
    P.g = io.g;
    if (ax == 0) {
      wire_in(P, io, true);
      P.e = e_of<T>(p);
    } else {
      P.in_a = chanA<T>(p);
      P.in_c = chanC<T>(p);
    }
    if (!P.last) {
      P.out_a = chanA<T>(p);
      P.out_c = chanC<T>(p);
    } else {
      wire_out(P, io);
      P.finish = finish;
      P.src = src;
      P.invmu = io.diag ? io.diag : invmu_of<T>(p);
      if (precond) P.post = d == 1 ? POST_DST_MU_DST : POST_DST;
    }
    TRY(enq(P, st));
  }
  if (precond && d > 1) TRY(enq_minv_tail<T>(p, st, io, d - 2, false));
  return TAU_OK;
}

// P_c^{-1} of the Strang circulant method: Hartley along dims d-1..1, Hartley·(1/p_c)·Hartley along
// dim 0, Hartley along 1..d-1 (the separable orthonormal Hartley transform is its own inverse and
// diagonalises every factor's Strang circulant), reading io's input and working in place after.
template <typename T>
tau_status enq_hartley(tau_problem* p, cudaStream_t st, const ChainT<T>& io) {
  bool rd = true;
  auto pass = [&](int ax, int post) -> tau_status {
    PassT<T> P = base_pass_t<T>(p, ax);
    P.post = post;
    P.invmu = reinterpret_cast<const T*>(p->pcinv);
    P.g = io.g;
    wire_in(P, io, rd);
    wire_out(P, io);
    rd = false;
    return enq(P, st);
  };
  for (int ax = p->d - 1; ax >= 1; --ax) TRY(pass(ax, POST_HT));
  TRY(pass(0, POST_HT_D_HT));
  for (int ax = 1; ax < p->d; ++ax) TRY(pass(ax, POST_HT));
  return TAU_OK;
}

template <typename T>
tau_status enq_minv(tau_problem* p, cudaStream_t st, const ChainT<T>& io) {
  return enq_minv_tail<T>(p, st, io, p->d - 1, true);
}

// Fields of the current step (from g->m): E, dt F in FP64, plus their copies in the element type
// of the solver (double-float: converted here; FP32 inner solve: e only).
tau_status enq_fields(tau_problem* p, cudaStream_t st, int64_t m_override) {
  KL(launch_fields(field_dev(p), p->g, m_override, p->E, p->Fdt, st));
  if (p->dfm) {
    KL(launch_d_to_df(p->E, p->Edf, p->n_tot, st));
    KL(launch_d_to_df(p->Fdt, p->Fdf, p->n_tot, st));
  }
  if (p->res_df) KL(launch_d_to_df(p->E, p->Edf, p->n_tot, st));
  if (p->mixed) KL(launch_f64_to_f32(p->E, p->E32, p->n_tot, st));
  return TAU_OK;
}

template <typename T> T* as(double* v) { return reinterpret_cast<T*>(v); }
template <typename T> const T* fdt_of(const tau_problem* p);
template <> const double* fdt_of<double>(const tau_problem* p) { return p->Fdt; }
template <> const df64* fdt_of<df64>(const tau_problem* p) { return p->Fdf; }

// Plain GMRES step in element type T (double, or double-float pairs stored in the same buffers).
template <typename T>
tau_status enq_prologue_t(tau_problem* p, cudaStream_t st) {
  TRY(enq_fields(p, st, -1));
  ChainT<T> rhs;
  rhs.x = as<T>(p->u);
  rhs.out = as<T>(p->b);
  TRY(enq_mv<T>(p, st, rhs, -1.0, FIN_ADD_F, fdt_of<T>(p), false));
  ChainT<T> r0;
  r0.out = as<T>(p->V);
  // two-sided: r_0 = P^{-1/2} B^{-1} (b - A u_0), the residual of Eq. (Pls) at ũ_0 = P^{1/2} u_0
  if (p->tpgm) r0.diag = as<T>(p->pmhb);
  // Strang circulant method: r_0 = P_c^{-1} B^{-1} (b - A u_0), B^{-1} on the sine basis
  if (p->spgm) r0.diag = as<T>(p->binv);
  if (p->desc.x0_mode == TAU_X0_PREV) {
    r0.x = as<T>(p->u);
    TRY(enq_mv<T>(p, st, r0, 1.0, FIN_RESID, as<T>(p->b), true));
  } else {
    r0.x = as<T>(p->b);
    TRY(enq_minv<T>(p, st, r0));
  }
  if (p->spgm) {
    ChainT<T> hc;
    hc.x = as<T>(p->V);
    hc.out = as<T>(p->V);
    TRY(enq_hartley<T>(p, st, hc));
  }
  KL(launch_norm_partial<T>(as<T>(p->V), p->n_tot, p->g, p->pnorm, st));
  tl_launches += 1;
  KL(launch_init_beta<T>(p->g, p->pnorm, p->gv, as<T>(p->V), p->n_tot, st));
  return TAU_OK;
}

template <typename T>
tau_status enq_body_t(tau_problem* p, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond) {
  ChainT<T> it;
  it.in_sel = 1;
  it.out_sel = 2;
  it.g = p->g;
  if (p->tpgm) {
    // two-sided operator of Eq. (Pls): v_{j+1} = P^{-1/2} B^{-1} A P^{-1/2} v_j, with P^{-1/2} v_j in tmp
    ChainT<T> half;
    half.in_sel = 1;
    half.out = as<T>(p->tmp);
    half.g = p->g;
    half.diag = as<T>(p->pmh);
    TRY(enq_minv<T>(p, st, half));
    it.in_sel = 0;
    it.x = as<T>(p->tmp);
    it.diag = as<T>(p->pmhb);
  }
  if (p->spgm) it.diag = as<T>(p->binv);
  TRY(enq_mv<T>(p, st, it, 1.0, FIN_NONE, nullptr, true));
  if (p->spgm) {
    // v_{j+1} = P_c^{-1} (B^{-1} A v_j), in place in the slot of v_{j+1}
    ChainT<T> hc;
    hc.in_sel = 2;
    hc.out_sel = 2;
    hc.g = p->g;
    TRY(enq_hartley<T>(p, st, hc));
  }
  const int ld = RED_BLOCKS;
  T* V = as<T>(p->V);
  KL(launch_dots<T>(V, p->n_tot, p->g, p->pdots, ld, p->h1, st));
  KL(launch_update_dots<T>(V, p->n_tot, p->g, p->h1, p->pdots, ld, p->h2, st));
  const GivensArgs ga{p->H, p->cs, p->sn, p->gv, p->h1, p->h2, p->desc.max_iter + 1, use_cond, h, nullptr};
  KL(launch_update_norm_givens<T>(V, p->n_tot, p->g, p->h2, p->pnorm, ga, st));
  KL(launch_scale_next<T>(V, p->n_tot, p->g, st));
  return TAU_OK;
}

template <typename T>
tau_status enq_epilogue_t(tau_problem* p, cudaStream_t st) {
  tl_launches += 2;
  if (p->tpgm) {
    // ũ = ũ_0 + V y and u = P^{-1/2} ũ = u_0 + P^{-1/2} (V y)
    KL(launch_backsolve_update<T>(p->g, p->H, p->gv, p->desc.max_iter + 1, p->y, as<T>(p->V), p->n_tot,
                                  as<T>(p->tmp), 0, p->iters, st));
    ChainT<T> half;
    half.x = as<T>(p->tmp);
    half.out = as<T>(p->A);
    half.diag = as<T>(p->pmh);
    TRY(enq_minv<T>(p, st, half));
    KL(launch_add_into(p->u, p->A, p->n_tot, p->desc.x0_mode == TAU_X0_PREV, st));
    return TAU_OK;
  }
  KL(launch_backsolve_update<T>(p->g, p->H, p->gv, p->desc.max_iter + 1, p->y, as<T>(p->V), p->n_tot, as<T>(p->u),
                                p->desc.x0_mode == TAU_X0_PREV, p->iters, st));
  return TAU_OK;
}

tau_status enq_prologue(tau_problem* p, cudaStream_t st) {
  return p->dfm ? enq_prologue_t<df64>(p, st) : enq_prologue_t<double>(p, st);
}
tau_status enq_body(tau_problem* p, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond) {
  return p->dfm ? enq_body_t<df64>(p, st, h, use_cond) : enq_body_t<double>(p, st, h, use_cond);
}

// ---- mixed precision: prologue, refinement sweep (before / after the inner loop), inner
//      FGMRES iteration, epilogue.  The refinement iterate X and the residual in tmp are FP64, or
//      double-float pairs in the same buffers when the residual runs on the FP32 pipes (res_df).
tau_status enq_mx_prologue(tau_problem* p, cudaStream_t st) {
  // b = (B E - S) u + dt F.  After a step, tmp holds r = b_old - A_old u and the flag is set:
  // then b = B((E_old + E)∘u) + r - b_old + dt F (a stencil, tau_mixed.cu) and the line passes of
  // the direct form skip themselves; otherwise (first step, a solution set by the caller) the
  // line passes run and the stencil kernels return at once.
  KL(launch_rres_save(p->rres, p->E, p->u, p->A, p->n_tot, st));
  TRY(enq_fields(p, st, -1));
  ChainIO rhs;
  rhs.x = p->u;
  rhs.out = p->b;
  TRY(enq_mv<double>(p, st, rhs, -1.0, FIN_ADD_F, p->Fdt, false, p->rres));
  {
    double bd[3] = {1.0, 1.0, 1.0}, bo[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < p->d; ++i) {
      bd[i] = 1.0 - p->desc.alpha[i] / 12.0;
      bo[i] = p->desc.alpha[i] / 24.0;
    }
    KL(launch_rres_rhs(p->rres, p->d, p->n, bd, bo, p->E, p->u, p->A, p->C, p->tmp, p->res_df ? 1 : 0, p->b,
                       p->Fdt, p->n_tot, st));
    tl_launches += p->d;   // 1 + d kernels
  }
  // (copies as kernels, so that a batch can record and group them; a zero double-float pair is
  // two zero floats, the bits of a zero double)
  if (p->res_df) {
    KL(launch_d_to_df(p->b, p->bdf, p->n_tot, st));
    if (p->desc.x0_mode == TAU_X0_PREV) KL(launch_d_to_df(p->u, as<df64>(p->X), p->n_tot, st));
    else KL(launch_copy(p->X, nullptr, p->n_tot, st));
  } else {
    KL(launch_copy(p->X, p->desc.x0_mode == TAU_X0_PREV ? p->u : nullptr, p->n_tot, st));
  }
  KL(launch_ir_init(p->ir, st));
  return TAU_OK;
}

tau_status enq_mx_sweep_pre(tau_problem* p, cudaStream_t st, cudaGraphConditionalHandle h,
                            cudaGraphConditionalHandle h_in, int use_cond) {
  // r = b - A x (FP64, or double-float); on the first sweep of a zero initial guess r = b and the
  // passes are skipped (the copy is bitwise, so it serves both storage types)
  const bool zero = p->desc.x0_mode == TAU_X0_ZERO;
  if (p->res_df) {
    KL(launch_ir_first_resid(p->ir, reinterpret_cast<const double*>(p->bdf), p->tmp, p->n_tot, zero, st));
    ChainT<df64> r;
    r.x = as<df64>(p->X);
    r.out = as<df64>(p->tmp);
    TRY(enq_mv<df64>(p, st, r, 1.0, FIN_RESID, p->bdf, false, &p->ir->skip_resid));
    KL(launch_norm_partial<df64>(as<df64>(p->tmp), p->n_tot, p->g, p->pnorm, st));
    KL(launch_ir_control(p->ir, p->gin, p->gvin, p->pnorm, p->n_tot, h, h_in, use_cond, p->gctl, st));
    KL(launch_scale_to_f32<df64>(as<df64>(p->tmp), p->V32, p->n_tot, p->ir, st));
    return TAU_OK;
  }
  KL(launch_ir_first_resid(p->ir, p->b, p->tmp, p->n_tot, zero, st));
  ChainIO r;
  r.x = p->X;
  r.out = p->tmp;
  TRY(enq_mv<double>(p, st, r, 1.0, FIN_RESID, p->b, false, &p->ir->skip_resid));
  KL(launch_norm_partial(p->tmp, p->n_tot, p->g, p->pnorm, st));
  KL(launch_ir_control(p->ir, p->gin, p->gvin, p->pnorm, p->n_tot, h, h_in, use_cond, p->gctl, st));
  KL(launch_scale_to_f32<double>(p->tmp, p->V32, p->n_tot, p->ir, st));
  return TAU_OK;
}

tau_status enq_mx_inner(tau_problem* p, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond) {
  // z_j = M^{-1} v_j (FP32), v_{j+1} = A z_j (FP32), CGS2, Givens: flexible GMRES
  ChainT<float> pz;
  pz.in_sel = 1;
  pz.in_base = p->V32;
  pz.out_sel = 1;
  pz.out_base = p->Z32;
  pz.g = p->gin;
  TRY(enq_minv<float>(p, st, pz));
  ChainT<float> av;
  av.in_sel = 1;
  av.in_base = p->Z32;
  av.out_sel = 2;
  av.out_base = p->V32;
  av.g = p->gin;
  TRY(enq_mv<float>(p, st, av, 1.0, FIN_NONE, nullptr, false));
  const int ld = RED_BLOCKS;
  KL(launch_dots<float>(p->V32, p->n_tot, p->gin, p->pdots, ld, p->h1in, st));
  KL(launch_update_dots<float>(p->V32, p->n_tot, p->gin, p->h1in, p->pdots, ld, p->h2in, st));
  const GivensArgs ga{p->Hin, p->csin, p->snin, p->gvin, p->h1in, p->h2in, p->kin + 1, use_cond, h,
                      p->gctl ? p->gctl + 1 : nullptr};
  KL(launch_update_norm_givens<float>(p->V32, p->n_tot, p->gin, p->h2in, p->pnorm, ga, st));
  KL(launch_scale_next<float>(p->V32, p->n_tot, p->gin, st));
  return TAU_OK;
}

tau_status enq_mx_sweep_post(tau_problem* p, cudaStream_t st) {
  KL(launch_backsolve(p->gin, p->Hin, p->gvin, p->kin + 1, p->yin, st));
  if (p->res_df) KL(launch_update_x<df64>(as<df64>(p->X), p->Z32, p->yin, p->n_tot, p->gin, p->ir, st));
  else KL(launch_update_x<double>(p->X, p->Z32, p->yin, p->n_tot, p->gin, p->ir, st));
  return TAU_OK;
}

tau_status enq_mx_epilogue(tau_problem* p, cudaStream_t st) {
  if (p->res_df) KL(launch_df_to_d(as<df64>(p->X), p->u, p->n_tot, st));
  else KL(launch_copy(p->u, p->X, p->n_tot, st));
  KL(launch_set_flag(p->rres, 1, st));   // tmp is the residual of this step's final iterate
  KL(launch_ir_finish(p->ir, p->g, p->iters, p->sweeps, st));
  return TAU_OK;
}

tau_status enq_epilogue(tau_problem* p, cudaStream_t st) {
  return p->dfm ? enq_epilogue_t<df64>(p, st) : enq_epilogue_t<double>(p, st);
}

// Record fn(stream) into graph g after deps; leaves receives the capture's final dependencies.
template <typename F>
tau_status capture_into(tau_problem* p, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, F fn,
                        std::vector<cudaGraphNode_t>& leaves) {
  CK(cudaStreamBeginCaptureToGraph(p->cap, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                   cudaStreamCaptureModeThreadLocal));
  tl_launches = 0;
  tau_status st = fn(p->cap);
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* d = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(p->cap, &cst, nullptr, nullptr, &d, nullptr, &nd);
  if (e == cudaSuccess) leaves.assign(d, d + nd);
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(p->cap, &out);
  if (st != TAU_OK) return st;
  if (e != cudaSuccess) return fail(TAU_EUNSUPPORTED, "capture info: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return fail(TAU_EUNSUPPORTED, "end capture: %s", cudaGetErrorString(e2));
  return TAU_OK;
}

// A conditional handle owned by g; its default value 1 is applied when the top-level graph is
// launched (not when an enclosing conditional body starts again).
tau_status make_handle(cudaGraph_t g, cudaGraphConditionalHandle* h) {
  cudaError_t e = cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail(TAU_EUNSUPPORTED, "conditional handle: %s", cudaGetErrorString(e));
  return TAU_OK;
}

// A conditional WHILE node after deps, driven by handle h (created on g).
tau_status add_while(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle* h,
                     cudaGraphNode_t* node, cudaGraph_t* body) {
  cudaError_t e;
  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  memset(cp_raw, 0, sizeof(cp_raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = *h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  e = cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &cp);
  if (e != cudaSuccess) return fail(TAU_EUNSUPPORTED, "conditional node: %s", cudaGetErrorString(e));
  *body = cp.conditional.phGraph_out[0];
  return TAU_OK;
}

// Plain step graph: prologue -> WHILE(GMRES iteration; the Givens kernel sets the condition) ->
// epilogue.  Mixed step graph: prologue -> WHILE(FP64 residual and refinement control ->
// WHILE(FP32 flexible GMRES iteration) -> correction of x) -> epilogue.
tau_status build_graph_inner(tau_problem* p, cudaGraph_t G) {
  std::vector<cudaGraphNode_t> none, leaves, tmp;
  if (!p->mixed) {
    TRY(capture_into(p, G, none, [&](cudaStream_t s) { return enq_prologue(p, s); }, leaves));
    p->k_pro = tl_launches;
    cudaGraphConditionalHandle h;
    cudaGraphNode_t w;
    cudaGraph_t body = nullptr;
    TRY(make_handle(G, &h));
    TRY(add_while(G, leaves, &h, &w, &body));
    TRY(capture_into(p, body, none, [&](cudaStream_t s) { return enq_body(p, s, h, 1); }, tmp));
    p->k_body = tl_launches;
    TRY(capture_into(p, G, {w}, [&](cudaStream_t s) { return enq_epilogue(p, s); }, tmp));
    p->k_epi = tl_launches;
    return TAU_OK;
  }
  TRY(capture_into(p, G, none, [&](cudaStream_t s) { return enq_mx_prologue(p, s); }, leaves));
  p->k_pro = tl_launches;
  cudaGraphConditionalHandle ho, hi;
  cudaGraphNode_t wo, wi;
  cudaGraph_t bo = nullptr, bi = nullptr;
  TRY(make_handle(G, &ho));
  TRY(add_while(G, leaves, &ho, &wo, &bo));
  TRY(make_handle(bo, &hi));
  std::vector<cudaGraphNode_t> pre;
  TRY(capture_into(p, bo, none, [&](cudaStream_t s) { return enq_mx_sweep_pre(p, s, ho, hi, 1); }, pre));
  p->k_ir_pre = tl_launches;
  TRY(add_while(bo, pre, &hi, &wi, &bi));
  TRY(capture_into(p, bi, none, [&](cudaStream_t s) { return enq_mx_inner(p, s, hi, 1); }, tmp));
  p->k_body = tl_launches;
  TRY(capture_into(p, bo, {wi}, [&](cudaStream_t s) { return enq_mx_sweep_post(p, s); }, tmp));
  p->k_ir_post = tl_launches;
  TRY(capture_into(p, G, {wo}, [&](cudaStream_t s) { return enq_mx_epilogue(p, s); }, tmp));
  p->k_epi = tl_launches;
  return TAU_OK;
}

tau_status build_graph(tau_problem* p) {
  cudaGraph_t G = nullptr;
  CK(cudaGraphCreate(&G, 0));
  tau_status st = build_graph_inner(p, G);
  if (st == TAU_OK) {
    cudaError_t e = cudaGraphInstantiate(&p->exec, G, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      st = fail(TAU_EUNSUPPORTED, "step graph: %s", cudaGetErrorString(e));
    }
  }
  cudaGraphDestroy(G);
  return st;
}

// Host-loop fallback: one synchronisation per GMRES iteration.
tau_status run_step_hostloop(tau_problem* p) {
  tl_launches = 0;
  TRY(enq_prologue(p, p->st));
  p->k_pro = tl_launches;
  cudaGraphConditionalHandle dummy = 0;
  for (int it = 0; it < p->desc.max_iter; ++it) {
    CK(cudaMemcpyAsync(p->h_done, &p->g->done, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    if (*p->h_done) break;
    tl_launches = 0;
    TRY(enq_body(p, p->st, dummy, 0));
    p->k_body = tl_launches;
  }
  tl_launches = 0;
  TRY(enq_epilogue(p, p->st));
  p->k_epi = tl_launches;
  return TAU_OK;
}

// Host-loop fallback of the mixed-precision step.
tau_status run_step_hostloop_mx(tau_problem* p) {
  cudaGraphConditionalHandle dummy = 0;
  tl_launches = 0;
  TRY(enq_mx_prologue(p, p->st));
  p->k_pro = tl_launches;
  for (int sw = 0; sw <= p->desc.max_sweeps + 1; ++sw) {
    tl_launches = 0;
    TRY(enq_mx_sweep_pre(p, p->st, dummy, dummy, 0));
    p->k_ir_pre = tl_launches;
    int flags[2];
    CK(cudaMemcpyAsync(&flags[0], &p->ir->done, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    if (flags[0]) break;
    for (int it = 0; it < p->kin; ++it) {
      CK(cudaMemcpyAsync(&flags[1], &p->gin->done, sizeof(int), cudaMemcpyDeviceToHost, p->st));
      CK(cudaStreamSynchronize(p->st));
      if (flags[1]) break;
      tl_launches = 0;
      TRY(enq_mx_inner(p, p->st, dummy, 0));
      p->k_body = tl_launches;
    }
    tl_launches = 0;
    TRY(enq_mx_sweep_post(p, p->st));
    p->k_ir_post = tl_launches;
  }
  tl_launches = 0;
  TRY(enq_mx_epilogue(p, p->st));
  p->k_epi = tl_launches;
  return TAU_OK;
}

// e and dt*F of step m into E / Fdt for the operator entry points (skipped when already there).
tau_status fields_for(tau_problem* p, int64_t m) {
  if (p->fields_m == m) return TAU_OK;
  TRY(enq_fields(p, p->st, m));
  p->fields_m = m;
  return TAU_OK;
}

// ---- tile autotuner: lines per CTA for each dimension and element type.  Candidates are timed
// on the real matvec pass (channels a, c in place) with CUDA events; results are cached per shape.
// ---- persistent record of the autotuner's decisions (lines per CTA, route, tensor cores), keyed
// by device and shape.  It lives in memory for the process and, unless TAU_TUNE_CACHE is "off",
// "0" or empty, in a text file: $TAU_TUNE_CACHE, else $XDG_CACHE_HOME/tau_rsfde/autotune.txt, else
// $HOME/.cache/tau_rsfde/autotune.txt.  The file's first line names the library build; a file
// written by another build is discarded (its kernels may have changed), so a rebuilt library
// measures again.  Lines are "key<TAB>value"; a later line overrides an earlier one.
struct TuneStore {
  std::mutex mu;
  bool loaded = false, fresh = true;   // fresh: the file must be (re)written with a header first
  std::string path;
  std::map<std::string, std::string> kv;
};
TuneStore g_store;

std::string tune_header() { return std::string("# tau_rsfde autotune ") + __DATE__ + " " + __TIME__; }

std::string tune_path() {
  const char* e = std::getenv("TAU_TUNE_CACHE");
  if (e) return (!e[0] || !strcmp(e, "off") || !strcmp(e, "0")) ? std::string() : std::string(e);
  const char* x = std::getenv("XDG_CACHE_HOME");
  std::string base;
  if (x && x[0]) {
    base = x;
  } else {
    const char* h = std::getenv("HOME");
    if (!h || !h[0]) return std::string();
    base = std::string(h) + "/.cache";
  }
  return base + "/tau_rsfde/autotune.txt";
}

void tune_load_locked() {
  if (g_store.loaded) return;
  g_store.loaded = true;
  g_store.path = tune_path();
  if (g_store.path.empty()) return;
  FILE* f = fopen(g_store.path.c_str(), "r");
  if (!f) return;
  char line[1024];
  const std::string hdr = tune_header();
  if (fgets(line, sizeof(line), f) && std::string(line).rfind(hdr, 0) == 0) {
    g_store.fresh = false;
    while (fgets(line, sizeof(line), f)) {
      std::string s(line);
      while (!s.empty() && (s.back() == '\n' || s.back() == '\r')) s.pop_back();
      const size_t t = s.find('\t');
      if (t != std::string::npos) g_store.kv[s.substr(0, t)] = s.substr(t + 1);
    }
  }
  fclose(f);
}

bool tune_get(const std::string& key, std::string* val) {
  std::lock_guard<std::mutex> lk(g_store.mu);
  tune_load_locked();
  auto it = g_store.kv.find(key);
  if (it == g_store.kv.end()) return false;
  *val = it->second;
  return true;
}

// Record a decision; the file write is best effort (a read-only cache location only costs a
// measurement in the next process).
void tune_put(const std::string& key, const std::string& val) {
  std::lock_guard<std::mutex> lk(g_store.mu);
  tune_load_locked();
  g_store.kv[key] = val;
  if (g_store.path.empty()) return;
  if (g_store.fresh) {
    for (size_t s = 1; (s = g_store.path.find('/', s)) != std::string::npos; ++s)
      mkdir(g_store.path.substr(0, s).c_str(), 0755);
    FILE* f = fopen(g_store.path.c_str(), "w");
    if (!f) return;
    fprintf(f, "%s\n", tune_header().c_str());
    for (const auto& e : g_store.kv) fprintf(f, "%s\t%s\n", e.first.c_str(), e.second.c_str());
    fclose(f);
    g_store.fresh = false;
    return;
  }
  FILE* f = fopen(g_store.path.c_str(), "a");
  if (!f) return;
  fprintf(f, "%s\t%s\n", key.c_str(), val.c_str());
  fclose(f);
}

// Device part of every key: name and SM count of the current device.
std::string dev_key() {
  int dev = 0;
  cudaDeviceProp pr{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string s = pr.name;
  for (char& ch : s)
    if (ch == ' ' || ch == '\t' || ch == '|') ch = '_';
  return s + "/" + std::to_string(pr.multiProcessorCount);
}

std::string join_key(std::initializer_list<long long> v) {
  std::string s;
  for (long long x : v) s += "|" + std::to_string(x);
  return s;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int64_t, int64_t>, int> g_tune_cache;

template <typename T>
tau_status tune_dim(tau_problem* p, int ax, T* chA, T* chC) {
  PassT<T> P = base_pass_t<T>(p, ax);   // heuristic tile (lpb_tuned not yet set for this axis)
  if (P.dim.route == ROUTE_LONG) {        // no line tiles on the long-line route
    p->lpb_tuned[prec_index<T>()][ax] = P.lpb;
    return TAU_OK;
  }
  const auto key = std::make_tuple(prec_index<T>(), P.dim.route, P.len, P.inner, P.nlines);
  const std::string skey = "lpb|" + dev_key() + join_key({prec_index<T>(), P.dim.route, P.len, P.inner, P.nlines});
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      p->lpb_tuned[prec_index<T>()][ax] = it->second;
      return TAU_OK;
    }
  }
  {
    std::string v;
    if (tune_get(skey, &v) && atoi(v.c_str()) > 0) {
      p->lpb_tuned[prec_index<T>()][ax] = atoi(v.c_str());
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = atoi(v.c_str());
      return TAU_OK;
    }
  }
  if (!p->tune_measure) return TAU_OK;   // recorded choices only: the heuristic stands
  // representative work: one matvec pass (channels a, c in place) and one DST pass (on c)
  P.seta = 1.0;
  P.in_a = chA;
  P.in_c = chC;
  P.out_a = chA;
  P.out_c = chC;
  PassT<T> Q = P;
  P.mv = 1;
  Q.post = POST_DST;
  Q.in_a = chC;
  Q.out_a = chC;
  const int heur = P.lpb;
  const int64_t cap = ax == 0 ? P.nlines : P.inner;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // candidates: lines per CTA (powers of two within 200 KB of shared memory) x threads per CTA
  // (128, or 256 for the wide variant); encoded lpb | (wide << 16)
  auto time_lpb = [&](int code, float* ms) -> tau_status {
    const int lpb = code & 0xFFFF;
    P.tpb = Q.tpb = (code >> 16) ? 256 : 128;
    set_lpb(P, lpb);
    set_lpb(Q, lpb);
    CK(launch_pass(P, p->st));
    CK(launch_pass(Q, p->st));
    CK(cudaEventRecord(e0, p->st));
    for (int r = 0; r < 3; ++r) {
      CK(launch_pass(P, p->st));
      CK(launch_pass(Q, p->st));
    }
    CK(cudaEventRecord(e1, p->st));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    return TAU_OK;
  };
  float best = 0.0f;
  TRY(time_lpb(heur, &best));
  int best_lpb = heur;
  for (int wide = 0; wide < 2; ++wide)
    for (int lpb = 1; lpb <= 32 && lpb <= cap; lpb *= 2) {
      if (lpb == heur && !wide) continue;
      set_lpb(P, lpb);
      if (pass_smem_bytes(P) > 200 * 1024) break;
      float ms = 0.0f;
      const int code = lpb | (wide << 16);
      TRY(time_lpb(code, &ms));
      if (ms < best * 0.97f) {
        best = ms;
        best_lpb = code;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->lpb_tuned[prec_index<T>()][ax] = best_lpb;
  tune_put(skey, std::to_string(best_lpb));
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best_lpb;
  return TAU_OK;
}

tau_status autotune(tau_problem* p) {
  CK(cudaMemsetAsync(p->A, 0, p->n_tot * sizeof(double), p->st));
  CK(cudaMemsetAsync(p->C, 0, p->n_tot * sizeof(double), p->st));
  for (int ax = 0; ax < p->d; ++ax) TRY(tune_dim<double>(p, ax, p->A, p->C));
  if (p->dfm || p->res_df)
    for (int ax = 0; ax < p->d; ++ax) TRY(tune_dim<df64>(p, ax, as<df64>(p->A), as<df64>(p->C)));
  if (p->mixed) {
    CK(cudaMemsetAsync(p->A32, 0, p->n_tot * sizeof(float), p->st));
    CK(cudaMemsetAsync(p->C32, 0, p->n_tot * sizeof(float), p->st));
    for (int ax = 0; ax < p->d; ++ax) TRY(tune_dim<float>(p, ax, p->A32, p->C32));
  }
  CK(cudaStreamSynchronize(p->st));
  return TAU_OK;
}

tau_status check_ready(tau_problem* p) {
  if (!p) return fail(TAU_EINVAL, "problem is NULL");
  if (!p->setup_done) return fail(TAU_ESTATE, "tau_setup has not run");
  return TAU_OK;
}

tau_status sync_status(tau_problem* p) {
  CK(cudaStreamSynchronize(p->st));
  if (p->tc_err) {
    // an expired wait is reported once: the flag is cleared with the report, so later syncs see
    // only waits that expire after it (the results of the work in flight at the time are not valid)
    int e = 0;
    CK(cudaMemcpy(&e, p->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
      CK(cudaMemset(p->tc_err, 0, sizeof(int)));
      return fail(TAU_ETIMEOUT, "a tensor-core pass gave up waiting on an mbarrier (its copies or MMAs)");
    }
  }
  GmresDev g;
  CK(cudaMemcpy(&g, p->g, sizeof(GmresDev), cudaMemcpyDeviceToHost));
  if (g.notconv) return fail(TAU_ENOTCONV, "a step reached max_iter=%d without meeting tol", p->desc.max_iter);
  return TAU_OK;
}

// LONG route tables of dimension i (d = 1): the four-step factorisation F = F1 x F2 of the
// convolution length F = 2 K_T, the stage and four-step twiddles, the Toeplitz circulant spectrum
// and the chirp-z kernel spectrum (both through the route's own forward transform, so they sit in
// its output layout), the chirp w_m, the scratch, and q on the device (Eq. (q), O(n^2) work).
tau_status setup_long(tau_problem* p, int i, const std::vector<double>& s) {
  const int N = p->n[i];
  int64_t kt = 2;
  while (kt < (int64_t)N + 1) kt <<= 1;
  const int F = (int)(2 * kt);
  int lgF = 0;
  while ((1 << lgF) < F) ++lgF;
  const int F1 = 1 << ((lgF + 1) / 2), F2 = F / F1;
  LongTab<double>& L = p->lt64[i];
  L.n = N;
  L.F = F;
  L.F1 = F1;
  L.F2 = F2;
  // one column per CTA and about F1/256 rows per CTA: at least 2 x 128 CTAs per launch where the
  // transform allows (with 128 CTAs on 152 SMs the launches ran at ~6 % occupancy, latency-bound)
  L.cw = 1;
  {
    int lpr = F1 / 256;
    if (lpr > 4096 / F2) lpr = 4096 / F2;
    if (lpr < 1) lpr = 1;
    L.lpr = lpr;
  }
  double2 *tw1 = nullptr, *tw2 = nullptr, *tw4 = nullptr, *lam = nullptr, *bh = nullptr, *w = nullptr;
  TRY(dalloc_n(p, &tw1, (size_t)twp_size(F1)));
  TRY(dalloc_n(p, &tw2, (size_t)twp_size(F2)));
  TRY(dalloc_n(p, &tw4, (size_t)F));
  TRY(dalloc_n(p, &lam, (size_t)F));
  TRY(dalloc_n(p, &bh, (size_t)F));
  KL(launch_twp(F1, tw1, p->st));
  KL(launch_twp(F2, tw2, p->st));
  KL(launch_long_tw4(F1, F2, tw4, p->st));
  double2* work = nullptr;
  double* ybuf = nullptr;
  TRY(dalloc_n(p, &work, (size_t)F));             // 16 bytes per entry: any element type's complex
  TRY(dalloc_n(p, &ybuf, 2 * (size_t)N));         // 16 bytes per entry: any element type
  L.tw1 = tw1;
  L.tw2 = tw2;
  L.tw4 = tw4;
  L.work = work;
  L.ybuf = ybuf;
  // chirp w_m = exp(i pi m^2/(2L)), m = 0..N (m^2 reduced mod 4L); kernel conj(w_|m|) at m mod F
  const int64_t Lc = (int64_t)N + 1;
  auto wph = [&](int64_t m) {
    const int64_t r = (m * m) % (4 * Lc);
    return make_double2(std::cos(M_PI * (double)r / (2.0 * (double)Lc)),
                        std::sin(M_PI * (double)r / (2.0 * (double)Lc)));
  };
  std::vector<double2> wv((size_t)N + 1), host((size_t)F, make_double2(0.0, 0.0));
  for (int m = 0; m <= N; ++m) wv[m] = wph(m);
  TRY(upload(p, &w, wv.data(), wv.size()));
  L.chirp = w;
  // q's cosine table ct[t] = cos(pi t / L), t < 2L, and q's storage (tracked allocations first)
  std::vector<double> ct(2 * (size_t)Lc);
  for (int64_t t = 0; t < 2 * Lc; ++t) ct[t] = std::cos(M_PI * (double)t / (double)Lc);
  double* dct = nullptr;
  TRY(upload(p, &dct, ct.data(), ct.size()));
  TRY(dalloc_n(p, &p->q[i], (size_t)N));
  double2* src = nullptr;   // untracked staging buffer, freed before returning
  CK(cudaMalloc(&src, (size_t)F * sizeof(double2)));
  auto release = [&](tau_status st) {
    cudaStreamSynchronize(p->st);
    cudaFree(src);
    src = nullptr;
    return st;
  };
  // Toeplitz: c_0 = s_0, c_k = c_{F-k} = s_k (1 <= k < N); spectrum / F
  host[0].x = s[0];
  for (int k = 1; k < N; ++k) host[k].x = host[(size_t)F - k].x = s[k];
  if (cudaMemcpy(src, host.data(), (size_t)F * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess)
    return release(fail(TAU_ECUDA, "long-route spectrum upload"));
  if (launch_long_spectrum(L, src, lam, 1.0 / F, p->st) != cudaSuccess)
    return release(fail(TAU_ECUDA, "long-route spectrum"));
  // chirp kernel: spectrum * sqrt(2/L) / F
  std::fill(host.begin(), host.end(), make_double2(0.0, 0.0));
  for (int m = -(N - 1); m <= N - 1; ++m) {
    const double2 v = wph(m < 0 ? -m : m);
    host[(size_t)(((int64_t)m % F + F) % F)] = make_double2(v.x, -v.y);
  }
  if (cudaStreamSynchronize(p->st) != cudaSuccess ||
      cudaMemcpy(src, host.data(), (size_t)F * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess)
    return release(fail(TAU_ECUDA, "long-route kernel upload"));
  if (launch_long_spectrum(L, src, bh, std::sqrt(2.0 / (double)Lc) / F, p->st) != cudaSuccess)
    return release(fail(TAU_ECUDA, "long-route kernel spectrum"));
  L.lam = lam;
  L.bhat = bh;
  if (launch_q_direct(N, p->s[i], dct, p->q[i], p->st) != cudaSuccess) return release(fail(TAU_ECUDA, "q"));
  return release(TAU_OK);
}

// The long-route tables of dimension i in another element type T (conv: double array -> T array
// on the device); the scratch buffers are shared with the FP64 tables (16 bytes per entry).
template <typename T, typename Conv>
tau_status long_tables_as(tau_problem* p, int i, LongTab<T>& D, int cw, Conv conv) {
  const LongTab<double>& L = p->lt64[i];
  D.n = L.n;
  D.F = L.F;
  D.F1 = L.F1;
  D.F2 = L.F2;
  D.cw = L.F2 < cw ? L.F2 : cw;
  D.lpr = L.lpr;
  auto cvt = [&](const double2* src, const vec2<T>** dst, size_t cnt) -> tau_status {
    T* f = nullptr;
    TRY(conv(reinterpret_cast<const double*>(src), &f, 2 * cnt));
    *dst = reinterpret_cast<const vec2<T>*>(f);
    return TAU_OK;
  };
  TRY(cvt(L.tw1, &D.tw1, (size_t)twp_size(L.F1)));
  TRY(cvt(L.tw2, &D.tw2, (size_t)twp_size(L.F2)));
  TRY(cvt(L.tw4, &D.tw4, (size_t)L.F));
  TRY(cvt(L.lam, &D.lam, (size_t)L.F));
  TRY(cvt(L.bhat, &D.bhat, (size_t)L.F));
  TRY(cvt(L.chirp, &D.chirp, (size_t)L.n + 1));
  D.work = reinterpret_cast<vec2<T>*>(L.work);
  D.ybuf = reinterpret_cast<T*>(L.ybuf);
  return TAU_OK;
}

// Tensor map of a table of `chunks` contiguous blocks of `chunk` FP32 values each (chunk a multiple of
// 256, base 16-byte aligned), seen as a 2-D tensor of rows of 256 values: a box of chunk / 256 rows is
// one block, which a tiled bulk copy (TMA) writes to shared memory unchanged.  The encoder is the
// driver's, reached through the runtime's entry-point query (no link to libcuda).
tau_status encode_chunk_map(CUtensorMap* map, const float* base, int chunk, int chunks) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!enc) return fail(TAU_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (chunk % 256 != 0 || chunk / 256 > 256 || chunks < 1 || (reinterpret_cast<uintptr_t>(base) & 15) != 0)
    return fail(TAU_EINVAL, "tensor map of %d blocks of %d values: blocks of 256..65536 values in multiples of 256, "
                "16-byte base", chunks, chunk);
  const cuuint64_t dim[2] = {256, (cuuint64_t)chunks * (chunk / 256)};
  const cuuint64_t stride[1] = {256 * 4};
  const cuuint32_t box[2] = {256, (cuuint32_t)(chunk / 256)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dim, stride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TAU_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return TAU_OK;
}

// Tensor-core DST tables of the mixed form (TAU_TC_AUTO): for every dimension with n <= 256 the first
// h = ceil(n/2) rows of the orthonormal DST-I matrix S[k][j] = sqrt(2/(n+1)) sin(pi (j+1)(k+1)/(n+1))
// (j k reduced mod 2(n+1)); the other rows follow from S[n-1-k][j] = (-1)^j S[k][j].  Rounded to TF32
// (nearest, ties away: the rounding the kernel applies to its inputs), zero padded to Nh rows (h
// rounded up to 16; 128 on dimension 0) and Kp16 = n rounded up to 16 columns.
tau_status setup_tc(tau_problem* p) {
  if (p->desc.tc == TAU_TC_OFF) return TAU_OK;
  for (int i = 0; i < p->d; ++i) {
    const int n = p->n[i];
    if (n > 256) continue;
    if (!p->tc_err) {
      TRY(dalloc_n(p, &p->tc_err, 1));
      CK(cudaMemsetAsync(p->tc_err, 0, sizeof(int), p->st));
    }
    TcTab& t = p->tc[i];
    t.n = n;
    // matvec: dimension 0 takes T as the A operand in tiles of 128 rows (accumulators 128 columns per
    // tile); the others take it as the B operand (N a multiple of 16)
    t.N = i == 0 ? (n + 127) & ~127 : (n + 15) & ~15;
    t.Kp16 = (n + 15) & ~15;
    t.nalloc = 32;
    while (t.nalloc < t.N) t.nalloc <<= 1;
    // DST: half of S, the A operand (128 rows) on dimension 0, else the B operand (Nh rows); two
    // accumulators (even and odd j) of 128 (dimension 0: lines) or Nh columns each
    const int h = (n + 1) / 2;
    t.Nh = i == 0 ? 128 : (h + 15) & ~15;
    const int acc_cols = i == 0 ? 128 : t.Nh;
    t.nalloc_h = 32;
    while (t.nalloc_h < 2 * acc_cols) t.nalloc_h <<= 1;
    // stored per K-chunk of 16 columns in the kernel's shared-memory layout (core matrices of 8
    // rows x 4 values: byte offset (k/8)*512 + (q/4)*128 + (k%8)*16 + (q%4)*4 within the chunk),
    // slot q of chunk c holding column j = 16c + 2q (q < 8: even j) or 16c + 2(q-8) + 1 (odd j)
    std::vector<float> S((size_t)t.Nh * t.Kp16, 0.0f);
    const double sc = std::sqrt(2.0 / (double)(n + 1));
    const int64_t L2 = 2 * ((int64_t)n + 1);
    for (int k = 0; k < h; ++k)
      for (int j = 0; j < n; ++j) {
        const int64_t r = ((int64_t)(j + 1) * (k + 1)) % L2;
        float v = (float)(sc * std::sin(M_PI * (double)r / (double)(n + 1)));
        uint32_t b;
        std::memcpy(&b, &v, 4);
        b = (b + 0x1000u) & ~0x1FFFu;   // keep 10 mantissa bits, round to nearest (ties away)
        std::memcpy(&v, &b, 4);
        const int c = j >> 4, jj = j & 15, q = (jj & 1) * 8 + (jj >> 1);
        const size_t off = (size_t)c * t.Nh * 16 + ((size_t)(k >> 3) * 512 + (q >> 2) * 128 + (k & 7) * 16 + (q & 3) * 4) / 4;
        S[off] = v;
      }
    float* dS = nullptr;
    TRY(upload(p, &dS, S.data(), S.size()));
    t.S = dS;
    TRY(encode_chunk_map(&t.tmS, dS, t.Nh * 16, t.Kp16 / 16));
    t.err = p->tc_err;
    p->tc_on[i] = true;
    // the Toeplitz factor T[k][j] = s_|k-j| split as T_hi + T_lo (each rounded to TF32 from the
    // FP64 weights), per K-chunk of 16 in the matvec kernel's layout
    std::vector<double> sw(n);
    CK(cudaMemcpy(sw.data(), p->s[i], n * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<float> Th((size_t)t.N * t.Kp16, 0.0f), Tl((size_t)t.N * t.Kp16, 0.0f);
    auto rna = [](float v) {
      uint32_t b;
      std::memcpy(&b, &v, 4);
      b = (b + 0x1000u) & ~0x1FFFu;
      std::memcpy(&v, &b, 4);
      return v;
    };
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j) {
        const double w = sw[k > j ? k - j : j - k];
        const float hi = rna((float)w), lo = rna((float)(w - (double)hi));
        const int c = j >> 4, jj = j & 15;
        const size_t off =
            (size_t)c * t.N * 16 + ((size_t)(k >> 3) * 512 + (jj >> 2) * 128 + (k & 7) * 16 + (jj & 3) * 4) / 4;
        Th[off] = hi;
        Tl[off] = lo;
      }
    float *dh = nullptr, *dl = nullptr;
    TRY(upload(p, &dh, Th.data(), Th.size()));
    TRY(upload(p, &dl, Tl.data(), Tl.size()));
    t.Thi = dh;
    t.Tlo = dl;
    TRY(encode_chunk_map(&t.tmThi, dh, t.N * 16, t.Kp16 / 16));
    TRY(encode_chunk_map(&t.tmTlo, dl, t.N * 16, t.Kp16 / 16));
  }
  bool all = true;
  for (int i = 0; i < p->d; ++i) all = all && p->tc_on[i];
  if (all) {
    if (p->d == 3) {
      TRY(dalloc_n(p, &p->A2, (size_t)p->n_tot));
      TRY(dalloc_n(p, &p->C2, (size_t)p->n_tot));
    }
    p->tcm = true;
  }
  return TAU_OK;
}

// TAU_TC_AUTO: time the FP32 τ solve with the tensor-core DST and with the line passes (CUDA events,
// after a warm-up) and keep the faster; results are cached per grid shape.
std::mutex g_tc_mu;
std::map<std::tuple<int, int, int, int>, bool> g_tc_cache;

tau_status choose_tc(tau_problem* p) {
  if (p->desc.tc != TAU_TC_AUTO) return TAU_OK;
  bool any = false;
  for (int i = 0; i < p->d; ++i) any = any || p->tc_on[i];
  if (!any) return TAU_OK;
  const auto key = std::make_tuple(p->d, p->n[0], p->d > 1 ? p->n[1] : 0, p->d > 2 ? p->n[2] : 0);
  const std::string shape = dev_key() + join_key({p->d, p->n[0], p->d > 1 ? p->n[1] : 0, p->d > 2 ? p->n[2] : 0,
                                                  p->route[0], p->route[1], p->route[2]});
  bool use = false, cached = false;
  {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    auto it = g_tc_cache.find(key);
    if (it != g_tc_cache.end()) {
      use = it->second;
      cached = true;
    }
  }
  if (!cached) {
    std::string v;
    if (tune_get("tc|" + shape, &v)) {
      use = v == "1";
      cached = true;
      std::lock_guard<std::mutex> lk(g_tc_mu);
      g_tc_cache[key] = use;
    }
  }
  if (!cached && !p->tune_measure) return TAU_OK;   // no record and no measurement: tensor cores where n <= 256
  if (!cached) {
    CK(cudaMemsetAsync(p->V32, 0, p->n_tot * sizeof(float), p->st));
    ChainT<float> io;
    io.x = p->V32;
    io.out = p->Z32;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto time_minv = [&](float* ms) -> tau_status {
      for (int r = 0; r < 2; ++r) TRY(enq_minv<float>(p, p->st, io));
      CK(cudaEventRecord(e0, p->st));
      for (int r = 0; r < 3; ++r) TRY(enq_minv<float>(p, p->st, io));
      CK(cudaEventRecord(e1, p->st));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(ms, e0, e1));
      return TAU_OK;
    };
    bool saved[3];
    for (int i = 0; i < 3; ++i) saved[i] = p->tc_on[i];
    float t_on = 0.0f, t_off = 0.0f;
    tau_status st = time_minv(&t_on);
    for (int i = 0; i < 3; ++i) p->tc_on[i] = false;
    if (st == TAU_OK) st = time_minv(&t_off);
    for (int i = 0; i < 3; ++i) p->tc_on[i] = saved[i];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TRY(st);
    use = t_on < 0.97f * t_off;
    tune_put("tc|" + shape, use ? "1" : "0");
    std::lock_guard<std::mutex> lk(g_tc_mu);
    g_tc_cache[key] = use;
  }
  if (!use)
    for (int i = 0; i < 3; ++i) p->tc_on[i] = false;
  if (p->tcm) {   // the split-TF32 matvec: its own measured choice
    const auto kmv = std::make_tuple(-p->d, p->n[0], p->d > 1 ? p->n[1] : 0, p->d > 2 ? p->n[2] : 0);
    bool use_mv = false, hit = false;
    {
      std::lock_guard<std::mutex> lk(g_tc_mu);
      auto it = g_tc_cache.find(kmv);
      if (it != g_tc_cache.end()) {
        use_mv = it->second;
        hit = true;
      }
    }
    if (!hit) {
      std::string v;
      if (tune_get("tcmv|" + shape, &v)) {
        use_mv = v == "1";
        hit = true;
        std::lock_guard<std::mutex> lk(g_tc_mu);
        g_tc_cache[kmv] = use_mv;
      }
    }
    if (!hit && !p->tune_measure) hit = use_mv = true;   // no record and no measurement: keep it
    if (!hit) {
      CK(cudaMemsetAsync(p->V32, 0, p->n_tot * sizeof(float), p->st));
      ChainT<float> io;
      io.x = p->V32;
      io.out = p->Z32;
      cudaEvent_t e0, e1;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      auto time_mv = [&](float* ms) -> tau_status {
        for (int r = 0; r < 2; ++r) TRY(enq_mv<float>(p, p->st, io, 1.0, FIN_NONE, nullptr, false));
        CK(cudaEventRecord(e0, p->st));
        for (int r = 0; r < 3; ++r) TRY(enq_mv<float>(p, p->st, io, 1.0, FIN_NONE, nullptr, false));
        CK(cudaEventRecord(e1, p->st));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        return TAU_OK;
      };
      float t_on = 0.0f, t_off = 0.0f;
      tau_status st = time_mv(&t_on);
      p->tcm = false;
      if (st == TAU_OK) st = time_mv(&t_off);
      p->tcm = true;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      TRY(st);
      use_mv = t_on < 0.97f * t_off;
      tune_put("tcmv|" + shape, use_mv ? "1" : "0");
      std::lock_guard<std::mutex> lk(g_tc_mu);
      g_tc_cache[kmv] = use_mv;
    }
    if (!use_mv) p->tcm = false;
  }
  return TAU_OK;
}

// Per-dimension tables of the line passes on dimension i for its current route p->route[i]: the
// DST weights, the Toeplitz circulant spectrum and twiddles (FFT and chirp routes), the chirp-z
// DST-I tables (chirp route), the long-line route's four-step tables; and the τ eigenvalues q of
// Eq. (q) (uploaded to p->q[i]; on the long-line route computed on the device).
tau_status route_tables(tau_problem* p, int i, const std::vector<double>& s) {
  const int N = p->n[i], K = N + 1;
  std::vector<double> q(N);
  {
    // dense route: sin(pi t / K), t = 0..2K-1; FFT route: the half-length DST's input weights
    // with the orthonormal scale folded in, (1/2) sqrt(2/K) sin(pi t / K), t = 0..K-1
    std::vector<double> st(2 * (size_t)K);
    const double hs = p->route[i] == ROUTE_FFT ? 0.5 * std::sqrt(2.0 / K) : 1.0;
    for (int t = 0; t < 2 * K; ++t) st[t] = hs * std::sin(M_PI * t / K);
    TRY(upload(p, &p->sintab[i], st.data(), st.size()));
  }
  const bool chirp = p->route[i] == ROUTE_CHIRP;
  const bool lng = p->route[i] == ROUTE_LONG;
  if (p->route[i] == ROUTE_FFT || chirp) {
    // Toeplitz product: circulant embedding c of length 2KK (KK = K on the FFT route, the power
    // of two >= n+1 on the chirp route): c_0 = s_0, c_k = c_{2KK-k} = s_k (1 <= k < N), zeros
    // elsewhere.  On the FFT route its real spectrum at k = 1..N is also the eigenvalues q_k of
    // tau(S) (Eq. (q)).
    const int KK = chirp ? p->KT[i] : K;
    TRY(dalloc_n(p, &p->twK[i], (size_t)twp_size(KK)));
    KL(launch_twp(KK, p->twK[i], p->st));
    if (!chirp) {
      TRY(dalloc_n(p, &p->twK2[i], (size_t)twp_size(K / 2)));
      KL(launch_twp(K / 2, p->twK2[i], p->st));
    }
    std::vector<double> c(2 * (size_t)KK, 0.0);
    c[0] = s[0];
    for (int k = 1; k < N; ++k) c[k] = c[2 * KK - k] = s[k];
    double *dc = nullptr, *dl = nullptr;
    TRY(upload(p, &dc, c.data(), c.size()));
    TRY(dalloc_n(p, &dl, (size_t)KK + 1));
    KL(launch_spectrum(KK, dc, dl, p->twK[i], p->st));
    std::vector<double> lam(KK + 1);
    CK(cudaMemcpyAsync(lam.data(), dl, (KK + 1) * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    std::vector<double2> spec(4 * (size_t)(KK / 2 + 1));
    for (int k = 0; k <= KK / 2; ++k) {
      double abcd[8];
      toep_pack_coeffs(lam[k], lam[KK - k], std::cos(M_PI * k / KK), -std::sin(M_PI * k / KK), KK, abcd);
      for (int r = 0; r < 4; ++r) spec[4 * (size_t)k + r] = make_double2(abcd[2 * r], abcd[2 * r + 1]);
    }
    TRY(upload(p, &p->spec[i], spec.data(), spec.size()));
    if (!chirp)
      for (int k = 1; k <= N; ++k) q[k - 1] = lam[k];
  }
  if (lng) TRY(setup_long(p, i, s));
  if (p->route[i] == ROUTE_DENSE || chirp) {
    // q_k = s_0 + 2 sum_j s_j cos(pi j k / K) (Eq. (q)) with a cosine table
    std::vector<double> ct(2 * (size_t)K);
    for (int t = 0; t < 2 * K; ++t) ct[t] = std::cos(M_PI * t / K);
    for (int k = 1; k <= N; ++k) {
      double acc = s[0];
      int64_t ph = 0;
      for (int j = 1; j < N; ++j) {
        ph += k;
        if (ph >= 2 * K) ph -= 2 * K;
        acc += 2.0 * s[j] * ct[ph];
      }
      q[k - 1] = acc;
    }
  }
  if (!lng) TRY(upload(p, &p->q[i], q.data(), q.size()));
  if (chirp) {
    // chirp-z DST-I tables (two lines per Bluestein DFT of length L = N+1): c_m = exp(-i pi m^2/L),
    // m = 0..N (m^2 reduced mod 2L, the period of the phase); kernel b_m = conj(c_|m|) for |m| <= N
    // placed at m mod MC (MC = power of two >= 2N; b_N and b_{-N} coincide when MC = 2N, with one
    // value); its FFT in fft_dif's order times sqrt(2/L)/(2 MC)
    const int MCi = p->MC[i];
    const int64_t L = N + 1;
    auto cph = [&](int64_t m) {
      const int64_t r = (m * m) % (2 * L);
      return make_double2(std::cos(M_PI * (double)r / (double)L), -std::sin(M_PI * (double)r / (double)L));
    };
    std::vector<double2> w(N + 1), bk(MCi, make_double2(0.0, 0.0));
    for (int m = 0; m <= N; ++m) w[m] = cph(m);
    for (int m = -N; m <= N; ++m) {
      const double2 v = cph(m < 0 ? -m : m);
      bk[((m % MCi) + MCi) % MCi] = make_double2(v.x, -v.y);
    }
    TRY(upload(p, &p->chirp[i], w.data(), w.size()));
    TRY(dalloc_n(p, &p->twM[i], (size_t)twp_size(MCi)));
    KL(launch_twp(MCi, p->twM[i], p->st));
    double2* db = nullptr;
    TRY(upload(p, &db, bk.data(), bk.size()));
    TRY(dalloc_n(p, &p->bhat[i], (size_t)MCi));
    KL(launch_chirp_spectrum(MCi, db, p->bhat[i], p->twM[i], std::sqrt(2.0 / (double)L) / (2.0 * MCi), p->st));
  }
  return TAU_OK;
}

// Whether one line of n values fits the line-pass kernel's 200 KB of shared memory on a route,
// for elements of esz bytes: the line plus its transform row (2K on the FFT route, 2 rows of 2 K_T
// on the chirp route, the line and its outputs on the dense route).
bool route_fits(int64_t n, int route, size_t esz) {
  const size_t nn = (size_t)n, npad = (nn + 1) & ~(size_t)1;
  size_t kt = 2;
  while (kt < nn + 1) kt <<= 1;
  const size_t rs = route == ROUTE_FFT ? 2 * (nn + 1) : (route == ROUTE_CHIRP ? 4 * kt : 2 * nn);
  return esz * (npad + rs) <= 200 * 1024;
}

void set_route(tau_problem* p, int i, int r) {
  p->route[i] = r;
  if (r == ROUTE_CHIRP) {
    int64_t kt = 2, mc = 2;
    while (kt < (int64_t)p->n[i] + 1) kt <<= 1;
    while (mc < 2 * (int64_t)p->n[i]) mc <<= 1;
    p->KT[i] = (int)kt;
    p->MC[i] = (int)mc;
  }
}

// Routes the measured choice considers for dimension i: only for TAU_ROUTE_AUTO in d >= 2 with the
// τ methods (1-D lines keep the long-line rule; the Strang method's Hartley passes are dense).  The
// FFT route where n + 1 is a power of two, else the chirp route, against the dense route.
std::vector<int> route_candidates(const tau_problem* p, int i) {
  std::vector<int> c;
  if (p->desc.route[i] != TAU_ROUTE_AUTO || p->d == 1 || p->spgm) return c;
  const int64_t n = p->n[i], K = n + 1;
  const size_t esz = p->dfm ? 16 : 8;
  if (is_pow2(K) && K >= 2 && K <= KMAX) c.push_back(ROUTE_FFT);
  else if (n < KMAX && route_fits(n, ROUTE_CHIRP, esz)) c.push_back(ROUTE_CHIRP);
  if (n <= 8192 && route_fits(n, ROUTE_DENSE, esz)) c.push_back(ROUTE_DENSE);
  return c;
}

// Device time of the FP64 line passes along dimension i on its current route: its lines per CTA
// chosen first (tune_dim), then one matvec pass and one DST pass, the unit tune_dim times too,
// five times after a warm-up (CUDA events; milliseconds per repetition).
tau_status time_route(tau_problem* p, int i, double* ms) {
  p->lpb_tuned[0][i] = 0;
  TRY(tune_dim<double>(p, i, p->A, p->C));
  PassT<double> P = base_pass_t<double>(p, i);
  P.seta = 1.0;
  P.mv = 1;
  P.in_a = P.out_a = p->A;
  P.in_c = P.out_c = p->C;
  PassT<double> Q = base_pass_t<double>(p, i);
  Q.post = POST_DST;
  Q.in_a = Q.out_a = p->C;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = launch_pass(P, p->st);
  if (e == cudaSuccess) e = launch_pass(Q, p->st);
  if (e == cudaSuccess) e = cudaEventRecord(e0, p->st);
  for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
    e = launch_pass(P, p->st);
    if (e == cudaSuccess) e = launch_pass(Q, p->st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, p->st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(TAU_ECUDA, "route timing: %s", cudaGetErrorString(e));
  *ms = t / 5.0;
  return TAU_OK;
}

// The measured route choice of dimension i (the GEMM-or-FFT decision of the FP64 passes: dense
// O(n) mode products against the FFT or chirp-z transforms): every candidate's tables are built and
// its passes timed, the fastest is kept (its tables built last), and the decision is recorded per
// device and shape.  Without tuning, or with one candidate, the rule of tau_create stands.
tau_status choose_route(tau_problem* p, int i, const std::vector<double>& s, bool tune) {
  const std::vector<int> cands = tune ? route_candidates(p, i) : std::vector<int>();
  if (cands.size() < 2) return route_tables(p, i, s);
  int64_t inner = 1;
  for (int l = 0; l < i; ++l) inner *= p->n[l];
  const std::string key = "route|" + dev_key() + join_key({p->dfm ? 2 : 0, i, p->n[i], inner, p->n_tot / p->n[i]});
  std::string v;
  if (p->tune_records && tune_get(key, &v)) {
    int r = 0;
    double ms = 0.0, alt = 0.0;
    if (sscanf(v.c_str(), "%d %lf %lf", &r, &ms, &alt) == 3 &&
        std::find(cands.begin(), cands.end(), r) != cands.end()) {
      set_route(p, i, r);
      p->route_src[i] = 2;
      p->route_ms[i] = ms;
      p->route_alt_ms[i] = alt;
      return route_tables(p, i, s);
    }
  }
  if (!p->tune_measure) return route_tables(p, i, s);   // no record: the rule stands
  CK(cudaMemsetAsync(p->A, 0, p->n_tot * sizeof(double), p->st));
  CK(cudaMemsetAsync(p->C, 0, p->n_tot * sizeof(double), p->st));
  double best = 0.0, alt = 0.0;
  int best_r = -1;
  for (int r : cands) {
    set_route(p, i, r);
    TRY(route_tables(p, i, s));
    double ms = 0.0;
    TRY(time_route(p, i, &ms));
    if (best_r < 0 || ms < best) {
      if (best_r >= 0) alt = best;
      best = ms;
      best_r = r;
    } else if (alt == 0.0 || ms < alt) {
      alt = ms;
    }
  }
  if (p->route[i] != best_r) {
    set_route(p, i, best_r);
    TRY(route_tables(p, i, s));
  }
  p->lpb_tuned[0][i] = 0;   // set again by autotune (from the cache tune_dim filled)
  p->route_src[i] = 1;
  p->route_ms[i] = best;
  p->route_alt_ms[i] = alt;
  char buf[96];
  snprintf(buf, sizeof(buf), "%d %.6g %.6g", best_r, best, alt);
  tune_put(key, buf);
  return TAU_OK;
}

}  // namespace

extern "C" {

const char* tau_last_error(void) { return g_err.c_str(); }

tau_status tau_create(const tau_problem_desc* desc, void* stream, tau_problem** out) {
  if (!desc || !out) return fail(TAU_EINVAL, "desc/out is NULL");
  *out = nullptr;
  const tau_problem_desc& D = *desc;
  if (D.d < 1 || D.d > 3) return fail(TAU_EINVAL, "d=%d outside 1..3", D.d);
  double ksum = 0;
  int64_t n_tot = 1;
  for (int i = 0; i < D.d; ++i) {
    if (D.n[i] < 1 || D.n[i] > (1 << 20)) return fail(TAU_EINVAL, "n[%d]=%lld outside 1..2^20", i, (long long)D.n[i]);
    if (!(D.alpha[i] > 1.0 && D.alpha[i] < 2.0)) return fail(TAU_EINVAL, "alpha[%d]=%g not in (1,2)", i, D.alpha[i]);
    if (!(D.kappa[i] >= 0.0)) return fail(TAU_EINVAL, "kappa[%d]=%g < 0", i, D.kappa[i]);
    if (!(D.R[i] > D.L[i])) return fail(TAU_EINVAL, "R[%d] <= L[%d]", i, i);
    ksum += D.kappa[i];
    n_tot *= D.n[i];
  }
  if (!(ksum > 0)) return fail(TAU_EINVAL, "sum of kappa must be > 0");
  if (!(D.T > 0) || D.M < 1) return fail(TAU_EINVAL, "T must be > 0 and M >= 1");
  if (!(D.tol > 0) || D.max_iter < 1 || D.max_iter > MAX_ITER_CAP)
    return fail(TAU_EINVAL, "tol must be > 0 and 1 <= max_iter <= %d", MAX_ITER_CAP);
  if (D.x0_mode != TAU_X0_ZERO && D.x0_mode != TAU_X0_PREV) return fail(TAU_EINVAL, "x0_mode %d", D.x0_mode);
  if (D.precision != TAU_FP64 && D.precision != TAU_MIXED && D.precision != TAU_DF64)
    return fail(TAU_EINVAL, "precision %d", D.precision);
  if (D.method != TAU_OPGM && D.method != TAU_TPGM && D.method != TAU_SPGM)
    return fail(TAU_EINVAL, "method %d", D.method);
  if (D.tc != TAU_TC_AUTO && D.tc != TAU_TC_OFF && D.tc != TAU_TC_ON) return fail(TAU_EINVAL, "tc %d", D.tc);
  if (D.autotune < TAU_TUNE_AUTO || D.autotune > TAU_TUNE_RECORDED) return fail(TAU_EINVAL, "autotune %d", D.autotune);
  if (D.method != TAU_OPGM && D.precision != TAU_FP64)
    return fail(TAU_EUNSUPPORTED, "the two-sided and Strang circulant methods run in TAU_FP64 only");
  if (D.precision == TAU_MIXED &&
      (D.refine_tol < 0 || D.inner_tol < 0 || D.inner_max_iter < 0 || D.inner_max_iter > MAX_ITER_CAP ||
       D.max_sweeps < 0))
    return fail(TAU_EINVAL, "mixed-precision parameters out of range");
  if (n_tot > (int64_t)1 << 31) return fail(TAU_EINVAL, "n_tot=%lld too large", (long long)n_tot);

  tau_problem* p = new (std::nothrow) tau_problem();
  if (!p) return fail(TAU_ENOMEM, "host allocation");
  p->desc = D;
  p->st = (cudaStream_t)stream;
  p->d = D.d;
  p->n_tot = n_tot;
  p->dt = D.T / (double)D.M;
  for (int i = 0; i < D.d; ++i) {
    p->n[i] = (int)D.n[i];
    p->h[i] = (D.R[i] - D.L[i]) / (double)(D.n[i] + 1);
    p->eta[i] = D.kappa[i] * p->dt / (2.0 * std::pow(p->h[i], D.alpha[i]));
    const int64_t K = D.n[i] + 1;
    int r = D.route[i];
    const bool fft_ok = is_pow2(K) && K >= 2 && K <= KMAX;
    // shared memory one line of the pass kernel needs on each route (the kernel's dynamic limit is
    // 200 KB): the line plus its transform row (2K on the FFT route, the data then 2 MC reals of
    // chirp-z work on the chirp route, the line and its outputs on the dense route)
    const size_t esz = D.precision == TAU_DF64 ? 16 : 8;
    const size_t nn = (size_t)D.n[i], npad = (nn + 1) & ~(size_t)1;
    size_t kt = 2, mc = 2;
    while (kt < nn + 1) kt <<= 1;
    while (mc < 2 * nn) mc <<= 1;   // chirp route: DST convolution length (2 kt, or kt for n = 2^p)
    // (chirp: rows of 2K_T reals allocated in pairs, so one line takes two rows)
    auto fits = [&](int route) {
      const size_t rs = route == TAU_ROUTE_FFT ? 2 * (nn + 1) : (route == TAU_ROUTE_CHIRP ? 4 * kt : 2 * nn);
      return esz * (npad + rs) <= 200 * 1024;
    };
    if (r == TAU_ROUTE_AUTO) {
      r = fft_ok ? TAU_ROUTE_FFT : (D.n[i] >= 128 && D.n[i] < KMAX ? TAU_ROUTE_CHIRP : TAU_ROUTE_DENSE);
      if (r == TAU_ROUTE_CHIRP && !fits(r)) r = TAU_ROUTE_DENSE;
      // one line (d = 1): a CTA per line leaves the GPU idle; the four-step route spreads the
      // transforms over the GPU and wins from n ~ 300 (measured; the FFT route keeps n + 1 <= 512)
      if (D.d == 1 && D.method != TAU_SPGM && D.n[i] >= 128 && !(fft_ok && D.n[i] < 512)) r = TAU_ROUTE_LONG;
    }
    if (r == TAU_ROUTE_LONG && (D.d != 1 || D.method == TAU_SPGM)) {
      delete p;
      return fail(TAU_EUNSUPPORTED, "the long-line route serves d = 1 with the tau methods (dim %d)", i);
    }
    if (r == TAU_ROUTE_CHIRP && D.n[i] >= KMAX) {
      delete p;
      return fail(TAU_EUNSUPPORTED, "chirp route limited to n < %d (dim %d, n=%lld)", KMAX, i, (long long)D.n[i]);
    }
    if (r == TAU_ROUTE_FFT && !fft_ok) {
      delete p;
      return fail(TAU_EUNSUPPORTED, "FFT route needs n+1 a power of two in [2, %d] (dim %d, n=%lld)", KMAX, i,
                  (long long)D.n[i]);
    }
    if (r == TAU_ROUTE_DENSE && D.n[i] > 8192) {
      delete p;
      return fail(TAU_EUNSUPPORTED, "dense route limited to n <= 8192 (dim %d, n=%lld)", i, (long long)D.n[i]);
    }
    if (r != TAU_ROUTE_FFT && r != TAU_ROUTE_DENSE && r != TAU_ROUTE_CHIRP && r != TAU_ROUTE_LONG) {
      delete p;
      return fail(TAU_EINVAL, "route[%d]=%d", i, D.route[i]);
    }
    if (r != TAU_ROUTE_LONG && !fits(r)) {
      delete p;
      return fail(TAU_EUNSUPPORTED, "one line of dim %d (n=%lld) does not fit in shared memory on route %d", i,
                  (long long)D.n[i], r);
    }
    p->route[i] = r == TAU_ROUTE_FFT     ? ROUTE_FFT
                  : r == TAU_ROUTE_CHIRP ? ROUTE_CHIRP
                  : r == TAU_ROUTE_LONG  ? ROUTE_LONG
                                         : ROUTE_DENSE;
    if (p->route[i] == ROUTE_CHIRP) {
      p->KT[i] = (int)kt;
      p->MC[i] = (int)mc;
    }
  }
  auto cleanup = [&](tau_status s) {
    tau_destroy(p);
    return s;
  };
  if (cudaError_t e = init_kernel_attributes(); e != cudaSuccess)
    return cleanup(fail(TAU_ECUDA, "kernel attributes: %s", cudaGetErrorString(e)));
  if (cudaError_t e = init_long_attributes(); e != cudaSuccess)
    return cleanup(fail(TAU_ECUDA, "kernel attributes: %s", cudaGetErrorString(e)));
  if (cudaError_t e = init_tc_attributes(); e != cudaSuccess)
    return cleanup(fail(TAU_ECUDA, "kernel attributes: %s", cudaGetErrorString(e)));
  if (cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking); e != cudaSuccess)
    return cleanup(fail(TAU_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
  p->mixed = D.precision == TAU_MIXED;
  p->dfm = D.precision == TAU_DF64;
  p->tpgm = D.method == TAU_TPGM;
  p->spgm = D.method == TAU_SPGM;
  if (p->mixed) {
    if (p->desc.refine_tol == 0) p->desc.refine_tol = 1e-10;
    if (p->desc.inner_max_iter == 0) p->desc.inner_max_iter = 30;
    if (p->desc.max_sweeps == 0) p->desc.max_sweeps = 10;
    if (p->desc.inner_tol == 0) p->desc.inner_tol = 1e-5;
    p->kin = p->desc.inner_max_iter;
  }
  const int mi = D.max_iter;
  const int rows = (p->mixed ? (p->kin > mi ? p->kin : mi) : mi) + 1;
  tau_status s = TAU_OK;
  const size_t n = (size_t)n_tot;
  if (!p->mixed && (s = dalloc_n(p, &p->V, (size_t)(mi + 1) * n))) return cleanup(s);
  if (p->mixed) {
    const int k = p->kin;
    if ((s = dalloc_n(p, &p->X, n)) || (s = dalloc_n(p, &p->V32, (size_t)(k + 1) * n)) ||
        (s = dalloc_n(p, &p->Z32, (size_t)k * n)) || (s = dalloc_n(p, &p->A32, n)) || (s = dalloc_n(p, &p->C32, n)) ||
        (s = dalloc_n(p, &p->invmu32, n)) || (s = dalloc_n(p, &p->E32, n)) ||
        (s = dalloc_n(p, &p->Hin, (size_t)(k + 1) * k)) ||
        (s = dalloc_n(p, &p->csin, k)) || (s = dalloc_n(p, &p->snin, k)) || (s = dalloc_n(p, &p->gvin, k + 1)) ||
        (s = dalloc_n(p, &p->h1in, k + 1)) || (s = dalloc_n(p, &p->h2in, k + 1)) || (s = dalloc_n(p, &p->yin, k + 1)) ||
        (s = dalloc_n(p, &p->gin, 1)) || (s = dalloc_n(p, &p->ir, 1)) || (s = dalloc_n(p, &p->sweeps, (size_t)D.M)) ||
        (s = dalloc_n(p, &p->rres, 1)))
      return cleanup(s);
    if (cudaMemset(p->rres, 0, sizeof(int)) != cudaSuccess) return cleanup(fail(TAU_ECUDA, "memset"));
    // double-float copies of e and b for the residual passes (used when tau_setup picks them)
    if ((s = dalloc_n(p, &p->Edf, n)) || (s = dalloc_n(p, &p->bdf, n))) return cleanup(s);
  }
  if (p->dfm && ((s = dalloc_n(p, &p->Edf, n)) || (s = dalloc_n(p, &p->Fdf, n)) ||
                 (s = dalloc_n(p, &p->invmu_df, n))))
    return cleanup(s);
  if (p->tpgm && ((s = dalloc_n(p, &p->pmh, n)) || (s = dalloc_n(p, &p->pmhb, n)))) return cleanup(s);
  if (p->spgm && ((s = dalloc_n(p, &p->pcinv, n)) || (s = dalloc_n(p, &p->binv, n)))) return cleanup(s);
  if ((s = dalloc_n(p, &p->u, n)) || (s = dalloc_n(p, &p->b, n)) ||
      (s = dalloc_n(p, &p->A, n)) || (s = dalloc_n(p, &p->C, n)) || (s = dalloc_n(p, &p->E, n)) ||
      (s = dalloc_n(p, &p->Fdt, n)) || (s = dalloc_n(p, &p->invmu, n)) || (s = dalloc_n(p, &p->tmp, n)) ||
      (s = dalloc_n(p, &p->H, (size_t)(mi + 1) * mi)) || (s = dalloc_n(p, &p->cs, mi)) ||
      (s = dalloc_n(p, &p->sn, mi)) || (s = dalloc_n(p, &p->gv, mi + 1)) || (s = dalloc_n(p, &p->h1, mi + 1)) ||
      (s = dalloc_n(p, &p->h2, mi + 1)) || (s = dalloc_n(p, &p->y, mi + 1)) ||
      (s = dalloc_n(p, &p->pdots, (size_t)rows * RED_BLOCKS)) || (s = dalloc_n(p, &p->pnorm, RED_BLOCKS)) ||
      (s = dalloc_n(p, &p->escan, 2 * RED_BLOCKS)) || (s = dalloc_n(p, &p->g, 1)) ||
      (s = dalloc_n(p, &p->iters, (size_t)D.M)))
    return cleanup(s);
  if ((s = dalloc_n(p, &p->tc_err, 1))) return cleanup(s);
  if (cudaMemset(p->tc_err, 0, sizeof(int)) != cudaSuccess) return cleanup(fail(TAU_ECUDA, "memset"));
  if (cudaMallocHost(&p->h_done, sizeof(int)) != cudaSuccess) {
    p->h_done = nullptr;
    return cleanup(fail(TAU_ENOMEM, "cudaMallocHost"));
  }
  if (cudaMemset(p->iters, 0, sizeof(int) * (size_t)D.M) != cudaSuccess) return cleanup(fail(TAU_ECUDA, "memset"));
  *out = p;
  return TAU_OK;
}

tau_status tau_set_fields(tau_problem* p, const tau_field* e, const tau_field* f, const tau_field* psi) {
  if (!p || !e || !f || !psi) return fail(TAU_EINVAL, "NULL argument");
  if (p->fields_set) return fail(TAU_ESTATE, "fields already set");
  const int64_t M = p->desc.M;
  if (e->n_times != M || f->n_times != M || psi->n_times != 1)
    return fail(TAU_EINVAL, "n_times must be M=%lld for e and f, 1 for psi", (long long)M);
  if (e->rank < 1 || f->rank < 0 || psi->rank < 0) return fail(TAU_EINVAL, "bad rank");
  const tau_field* fs[3] = {e, f, psi};
  for (auto* fl : fs) {
    if (fl->rank > 0 && !fl->time_coef) return fail(TAU_EINVAL, "time_coef NULL");
    for (int i = 0; i < p->d; ++i)
      if (fl->rank > 0 && !fl->space[i]) return fail(TAU_EINVAL, "space[%d] NULL", i);
  }
  p->re = e->rank;
  p->rf = f->rank;
  p->rp = psi->rank;
  TRY(upload(p, &p->e_tc, e->time_coef, (size_t)M * e->rank));
  TRY(upload(p, &p->f_tc, f->time_coef, (size_t)M * f->rank));
  TRY(upload(p, &p->psi_tc, psi->time_coef, (size_t)psi->rank));
  for (int i = 0; i < p->d; ++i) {
    const int ni = p->n[i];
    TRY(upload(p, &p->e_sp[i], e->space[i], (size_t)e->rank * (ni + 2)));
    TRY(upload(p, &p->psi_sp[i], psi->space[i], (size_t)psi->rank * (ni + 2)));
    // F = (⊗ 𝓗_{alpha_l}) f restricted to the interior (Eq. (2.2) applied to the source; the
    // 1-D and 2-D forms of Appendix A): for separable f each factor takes the 3-point stencil.
    const double a = p->desc.alpha[i];
    std::vector<double> hs((size_t)f->rank * ni);
    for (int r = 0; r < f->rank; ++r) {
      const double* sp = f->space[i] + (size_t)r * (ni + 2);
      for (int j = 0; j < ni; ++j)
        hs[(size_t)r * ni + j] = (a / 24.0) * sp[j] + (1.0 - a / 12.0) * sp[j + 1] + (a / 24.0) * sp[j + 2];
    }
    TRY(upload(p, &p->f_hsp[i], hs.data(), hs.size()));
  }
  p->fields_set = true;
  return TAU_OK;
}

tau_status tau_set_fields_device(tau_problem* p, const tau_field_device* fd) {
  if (!p || !fd) return fail(TAU_EINVAL, "NULL argument");
  if (p->fields_set) return fail(TAU_ESTATE, "fields already set");
  if (!fd->e) return fail(TAU_EINVAL, "e is NULL (a coefficient field is required)");
  int64_t n_pad = 1;
  for (int i = 0; i < p->d; ++i) n_pad *= (int64_t)p->n[i] + 2;
  if (fd->e_step != 0 && fd->e_step != p->n_tot)
    return fail(TAU_EINVAL, "e_step=%lld must be 0 or n_tot=%lld", (long long)fd->e_step, (long long)p->n_tot);
  if (fd->f && fd->f_step != 0 && fd->f_step != n_pad)
    return fail(TAU_EINVAL, "f_step=%lld must be 0 or prod(n_i+2)=%lld", (long long)fd->f_step, (long long)n_pad);
  p->e_dev = fd->e;
  p->e_step = fd->e_step;
  p->f_dev = fd->f;
  p->f_step = fd->f ? fd->f_step : 0;
  p->psi_dev = fd->psi;
  p->re = p->rf = p->rp = 0;
  p->fields_set = true;
  return TAU_OK;
}

tau_status tau_setup(tau_problem* p) {
  if (!p) return fail(TAU_EINVAL, "problem is NULL");
  if (!p->fields_set) return fail(TAU_ESTATE, "neither tau_set_fields nor tau_set_fields_device has run");
  if (p->setup_done) return fail(TAU_ESTATE, "tau_setup already ran");
  const int d = p->d;
  // measured choices (routes, lines per CTA, tensor cores) for problems of >= 65536 unknowns, or
  // as TAU_AUTOTUNE says (1: always, 0: never; the rules of tau_create and the heuristics stand)
  if (p->desc.autotune == TAU_TUNE_AUTO) {
    const char* tn = std::getenv("TAU_AUTOTUNE");
    p->tune_measure = p->tune_records = tn ? tn[0] == '1' : p->n_tot >= (1 << 16);
  } else {
    p->tune_measure = p->desc.autotune == TAU_TUNE_ON;
    p->tune_records = p->desc.autotune == TAU_TUNE_ON || p->desc.autotune == TAU_TUNE_RECORDED;
  }
  const bool tune = p->tune_measure || p->tune_records;
  for (int i = 0; i < d; ++i) {
    const int N = p->n[i], K = N + 1;
    const double a = p->desc.alpha[i];
    // FCD weights by the recurrence of §2: s_0 = Gamma(a+1)/Gamma(a/2+1)^2,
    // s_k = (1 - (a+1)/(a/2+k)) s_{k-1}.
    std::vector<double> s(N);
    s[0] = std::tgamma(a + 1.0) / (std::tgamma(a / 2.0 + 1.0) * std::tgamma(a / 2.0 + 1.0));
    for (int k = 1; k < N; ++k) s[k] = (1.0 - (a + 1.0) / (a / 2.0 + k)) * s[k - 1];
    TRY(upload(p, &p->s[i], s.data(), s.size()));
    // eigenvalues of B_{alpha_i} on sine mode k = 1..N (Lemma Heig)
    std::vector<double> beta(N);
    for (int k = 1; k <= N; ++k) {
      const double sn = std::sin(k * M_PI / (2.0 * N + 2.0));
      beta[k - 1] = 1.0 - (a / 6.0) * sn * sn;
    }
    TRY(upload(p, &p->beta[i], beta.data(), beta.size()));
    if (p->spgm) {
      // Strang circulants of B_{alpha_i} and S_{alpha_i} (first column t, entries k > N/2 wrapped to
      // t_{N-k}) and their DFT eigenvalues lambda_m = sum_k c_k cos(2 pi k m / N) (real: symmetric);
      // the orthonormal Hartley table cas(2 pi t / N) / sqrt(N)
      std::vector<double> tb(N, 0.0);
      tb[0] = 1.0 - a / 12.0;
      if (N > 1) tb[1] = a / 24.0;
      auto strang = [&](const std::vector<double>& t) {
        std::vector<double> c(t);
        for (int k = N / 2 + 1; k < N; ++k) c[k] = t[N - k];
        return c;
      };
      const std::vector<double> cb = strang(tb), cs = strang(s);
      std::vector<double> cosN(N), lb(N), ls(N), ct(N);
      for (int t = 0; t < N; ++t) cosN[t] = std::cos(2.0 * M_PI * t / N);
      for (int m = 0; m < N; ++m) {
        double xb = 0.0, xs = 0.0;
        int ph = 0;
        for (int k = 0; k < N; ++k) {
          xb += cb[k] * cosN[ph];
          xs += cs[k] * cosN[ph];
          ph += m;
          if (ph >= N) ph -= N;
        }
        lb[m] = xb;
        ls[m] = xs;
      }
      for (int t = 0; t < N; ++t) ct[t] = (cosN[t] + std::sin(2.0 * M_PI * t / N)) / std::sqrt((double)N);
      TRY(upload(p, &p->sb[i], lb.data(), lb.size()));
      TRY(upload(p, &p->ss[i], ls.data(), ls.size()));
      TRY(upload(p, &p->cas[i], ct.data(), ct.size()));
    }
    TRY(choose_route(p, i, s, tune));
  }
  // ebar (Eqs. (bard), (dhat))
  if (std::isnan(p->desc.e_min) || std::isnan(p->desc.e_max)) {
    KL(launch_escan(field_dev(p), p->desc.M, p->escan, p->st));
    std::vector<double> part(2 * RED_BLOCKS);
    CK(cudaMemcpyAsync(part.data(), p->escan, part.size() * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    double hi = -INFINITY, lo = INFINITY;
    for (int b = 0; b < RED_BLOCKS; ++b) {
      hi = std::fmax(hi, part[2 * b]);
      lo = std::fmin(lo, part[2 * b + 1]);
    }
    p->ehat = hi;
    p->echeck = lo;
  } else {
    p->ehat = p->desc.e_max;
    p->echeck = p->desc.e_min;
  }
  if (!(p->echeck > 0.0) || !(p->ehat >= p->echeck))
    return fail(TAU_EINVAL, "e must be positive: min %g max %g", p->echeck, p->ehat);
  p->ebar = 0.5 * (p->ehat + p->echeck);
  KL(launch_invmu(d, p->n, p->n_tot, p->ebar, p->beta, p->q, p->eta, p->invmu, p->st));
  if (p->tpgm) KL(launch_tpgm_diag(d, p->n, p->n_tot, p->ebar, p->beta, p->q, p->eta, p->pmh, p->pmhb, p->st));
  if (p->spgm)
    KL(launch_spgm_diag(d, p->n, p->n_tot, p->ebar, p->sb, p->ss, p->eta, p->beta, p->pcinv, p->binv, p->st));
  if (p->e_dev) {
    double* u0 = p->dfm ? p->tmp : p->u;
    if (p->psi_dev) CK(cudaMemcpyAsync(u0, p->psi_dev, p->n_tot * sizeof(double), cudaMemcpyDeviceToDevice, p->st));
    else CK(cudaMemsetAsync(u0, 0, p->n_tot * sizeof(double), p->st));
  } else {
    KL(launch_psi(d, p->n, p->n_tot, p->rp, p->psi_tc, p->psi_sp, p->dfm ? p->tmp : p->u, p->st));
  }
  if (p->dfm) KL(launch_d_to_df(p->tmp, as<df64>(p->u), p->n_tot, p->st));
  if (p->mixed) {
    // The mixed form's outer residual b - A x runs as double-float line passes when their rounding
    // floor stays below half the refinement tolerance.  The cancelling Toeplitz sums of A x carry
    // an absolute error of about eps_df * (a few) * max_i eta_i ||s^{(i)}||_1 |x| (eps_df = 2^-48,
    // ||s||_1 <= 2 s_0, Eq. (As1)), against ||b|| ~ ebar |x|: floor = 2^-48 * 8 * max_i eta_i 2 s_0 / ebar.
    // Otherwise (large eta: long lines at alpha near 2) the residual stays FP64.
    double worst = 0.0;
    for (int i = 0; i < d; ++i) {
      const double a = p->desc.alpha[i], g = std::tgamma(a / 2.0 + 1.0);
      worst = std::max(worst, p->eta[i] * 2.0 * std::tgamma(a + 1.0) / (g * g));
    }
    p->res_df = std::ldexp(8.0 * worst / p->ebar, -48) <= 0.5 * p->desc.refine_tol;
  }
  if (p->dfm || p->res_df) {
    auto conv = [&](const double* src, df64** dst, size_t cnt) -> tau_status {
      TRY(dalloc_n(p, dst, cnt));
      KL(launch_d_to_df(src, *dst, (int64_t)cnt, p->st));
      return TAU_OK;
    };
    for (int i = 0; i < d; ++i) {
      const int N = p->n[i], K = N + 1;
      TRY(conv(p->s[i], &p->s_df[i], N));
      TRY(conv(p->sintab[i], &p->sintab_df[i], 2 * (size_t)K));
      if (p->route[i] == ROUTE_FFT || p->route[i] == ROUTE_CHIRP) {
        const int KK = p->route[i] == ROUTE_CHIRP ? p->KT[i] : K;
        df64* f = nullptr;
        TRY(conv(reinterpret_cast<const double*>(p->spec[i]), &f, 8 * (size_t)(KK / 2 + 1)));
        p->spec_df[i] = reinterpret_cast<df64x2*>(f);
        TRY(conv(reinterpret_cast<const double*>(p->twK[i]), &f, 2 * (size_t)twp_size(KK)));
        p->twK_df[i] = reinterpret_cast<df64x2*>(f);
      }
      if (p->route[i] == ROUTE_FFT) {
        df64* f = nullptr;
        TRY(conv(reinterpret_cast<const double*>(p->twK2[i]), &f, 2 * (size_t)twp_size(K / 2)));
        p->twK2_df[i] = reinterpret_cast<df64x2*>(f);
      }
      if (p->route[i] == ROUTE_CHIRP) {
        df64* f = nullptr;
        TRY(conv(reinterpret_cast<const double*>(p->chirp[i]), &f, 2 * (size_t)(N + 1)));
        p->chirp_df[i] = reinterpret_cast<df64x2*>(f);
        TRY(conv(reinterpret_cast<const double*>(p->bhat[i]), &f, 2 * (size_t)p->MC[i]));
        p->bhat_df[i] = reinterpret_cast<df64x2*>(f);
        TRY(conv(reinterpret_cast<const double*>(p->twM[i]), &f, 2 * (size_t)twp_size(p->MC[i])));
        p->twM_df[i] = reinterpret_cast<df64x2*>(f);
      }
      if (p->route[i] == ROUTE_LONG) TRY(long_tables_as(p, i, p->ltdf[i], 1, conv));
    }
    if (p->dfm) KL(launch_d_to_df(p->invmu, p->invmu_df, p->n_tot, p->st));
  }
  if (p->mixed) {
    auto conv = [&](const double* src, float** dst, size_t cnt) -> tau_status {
      TRY(dalloc_n(p, dst, cnt));
      KL(launch_f64_to_f32(src, *dst, (int64_t)cnt, p->st));
      return TAU_OK;
    };
    for (int i = 0; i < d; ++i) {
      const int N = p->n[i], K = N + 1;
      TRY(conv(p->s[i], &p->s32[i], N));
      TRY(conv(p->sintab[i], &p->sintab32[i], 2 * (size_t)K));
      if (p->route[i] == ROUTE_FFT || p->route[i] == ROUTE_CHIRP) {
        const int KK = p->route[i] == ROUTE_CHIRP ? p->KT[i] : K;
        float* f = nullptr;
        TRY(conv(reinterpret_cast<const double*>(p->spec[i]), &f, 8 * (size_t)(KK / 2 + 1)));
        p->spec32[i] = reinterpret_cast<float2*>(f);
        TRY(conv(reinterpret_cast<const double*>(p->twK[i]), &f, 2 * (size_t)twp_size(KK)));
        p->twK32[i] = reinterpret_cast<float2*>(f);
      }
      if (p->route[i] == ROUTE_FFT) {
        float* f = nullptr;
        TRY(conv(reinterpret_cast<const double*>(p->twK2[i]), &f, 2 * (size_t)twp_size(K / 2)));
        p->twK2_32[i] = reinterpret_cast<float2*>(f);
      }
      if (p->route[i] == ROUTE_CHIRP) {
        float* f = nullptr;
        TRY(conv(reinterpret_cast<const double*>(p->chirp[i]), &f, 2 * (size_t)(N + 1)));
        p->chirp32[i] = reinterpret_cast<float2*>(f);
        TRY(conv(reinterpret_cast<const double*>(p->bhat[i]), &f, 2 * (size_t)p->MC[i]));
        p->bhat32[i] = reinterpret_cast<float2*>(f);
        TRY(conv(reinterpret_cast<const double*>(p->twM[i]), &f, 2 * (size_t)twp_size(p->MC[i])));
        p->twM32[i] = reinterpret_cast<float2*>(f);
      }
      if (p->route[i] == ROUTE_LONG) TRY(long_tables_as(p, i, p->lt32[i], 1, conv));
    }
    KL(launch_f64_to_f32(p->invmu, p->invmu32, p->n_tot, p->st));
    TRY(setup_tc(p));
    TRY(choose_tc(p));
    IRDev ir{};
    ir.tol = p->desc.refine_tol;
    ir.max_sweeps = p->desc.max_sweeps;
    ir.inner_tol = p->desc.inner_tol;
    CK(cudaMemcpyAsync(p->ir, &ir, sizeof(ir), cudaMemcpyHostToDevice, p->st));
    GmresDev gi{};
    gi.max_iter = p->kin;
    gi.tol = p->desc.inner_tol;
    gi.done = 1;
    CK(cudaMemcpyAsync(p->gin, &gi, sizeof(gi), cudaMemcpyHostToDevice, p->st));
    CK(cudaMemsetAsync(p->sweeps, 0, sizeof(int) * (size_t)p->desc.M, p->st));
  }
  GmresDev g{};
  g.max_iter = p->desc.max_iter;
  g.tol = p->desc.tol;
  g.M = p->desc.M;
  g.m = 0;
  g.done = 1;
  CK(cudaMemcpyAsync(p->g, &g, sizeof(g), cudaMemcpyHostToDevice, p->st));
  CK(cudaStreamSynchronize(p->st));
  p->m_host = 0;
  if (tune) TRY(autotune(p));
  p->setup_done = true;
  const char* nog = std::getenv("TAU_NO_GRAPH");
  if (!(nog && nog[0] == '1')) {
    tau_status gs = build_graph(p);
    p->graph_ok = gs == TAU_OK;
    if (!p->graph_ok) g_err.clear();
  }
  return TAU_OK;
}

tau_status tau_step(tau_problem* p, int64_t count) {
  TRY(check_ready(p));
  if (count < 0 || p->m_host + count > p->desc.M)
    return fail(TAU_EINVAL, "count=%lld with m=%lld of M=%lld", (long long)count, (long long)p->m_host,
                (long long)p->desc.M);
  if (count > 0) p->fields_m = -1;
  for (int64_t c = 0; c < count; ++c) {
    if (p->graph_ok) {
      CK(cudaGraphLaunch(p->exec, p->st));
    } else if (p->mixed) {
      TRY(run_step_hostloop_mx(p));
    } else {
      TRY(run_step_hostloop(p));
    }
    ++p->m_host;
  }
  return TAU_OK;
}

tau_status tau_sync(tau_problem* p) {
  TRY(check_ready(p));
  return sync_status(p);
}

tau_status tau_solve(tau_problem* p) {
  TRY(check_ready(p));
  TRY(tau_step(p, p->desc.M - p->m_host));
  return sync_status(p);
}

tau_status tau_get_solution(tau_problem* p, double* out, int is_device, int64_t* m_out) {
  TRY(check_ready(p));
  if (!out) return fail(TAU_EINVAL, "out is NULL");
  const double* src = p->u;
  if (p->dfm) {
    KL(launch_df_to_d(as<df64>(p->u), p->tmp, p->n_tot, p->st));
    src = p->tmp;
  }
  CK(cudaMemcpyAsync(out, src, p->n_tot * sizeof(double), is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     p->st));
  if (!is_device) CK(cudaStreamSynchronize(p->st));
  if (m_out) *m_out = p->m_host;
  return TAU_OK;
}

tau_status tau_set_solution(tau_problem* p, const double* u, int is_device, int64_t m) {
  TRY(check_ready(p));
  if (!u) return fail(TAU_EINVAL, "u is NULL");
  if (m < 0 || m > p->desc.M) return fail(TAU_EINVAL, "m=%lld outside 0..M", (long long)m);
  CK(cudaMemcpyAsync(p->dfm ? p->tmp : p->u, u, p->n_tot * sizeof(double),
                     is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->st));
  if (p->dfm) KL(launch_d_to_df(p->tmp, as<df64>(p->u), p->n_tot, p->st));
  // m lives in the device state read by the step graph
  CK(cudaMemcpyAsync(&p->g->m, &m, sizeof(int64_t), cudaMemcpyHostToDevice, p->st));
  // the last residual no longer belongs to the solution: the next right-hand side takes the passes
  if (p->rres) CK(cudaMemsetAsync(p->rres, 0, sizeof(int), p->st));
  CK(cudaStreamSynchronize(p->st));
  p->m_host = m;
  return TAU_OK;
}

tau_status tau_get_stats(tau_problem* p, tau_stats* out) {
  TRY(check_ready(p));
  if (!out) return fail(TAU_EINVAL, "out is NULL");
  CK(cudaStreamSynchronize(p->st));
  GmresDev g;
  CK(cudaMemcpy(&g, p->g, sizeof(GmresDev), cudaMemcpyDeviceToHost));
  std::vector<int> it((size_t)p->desc.M);
  CK(cudaMemcpy(it.data(), p->iters, it.size() * sizeof(int), cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof(*out));
  out->steps_done = g.m;
  int64_t tot = 0;
  int mx = 0;
  for (int64_t m = 0; m < g.m && m < p->desc.M; ++m) {
    tot += it[m];
    if (it[m] > mx) mx = it[m];
  }
  out->total_iters = tot;
  out->last_iters = g.m > 0 ? it[g.m - 1] : 0;
  out->max_iters_step = mx;
  out->last_relres = g.relres;
  out->ebar = p->ebar;
  out->e_hat = p->ehat;
  out->e_check = p->echeck;
  for (int i = 0; i < 3; ++i) {
    const int r = i < p->d ? p->route[i] : 0;
    out->route[i] = r == ROUTE_FFT     ? TAU_ROUTE_FFT
                    : r == ROUTE_CHIRP ? TAU_ROUTE_CHIRP
                    : r == ROUTE_LONG  ? TAU_ROUTE_LONG
                    : r == ROUTE_DENSE ? TAU_ROUTE_DENSE
                                       : 0;
  }
  out->graph = p->graph_ok ? 1 : 0;
  for (int i = 0; i < 3; ++i) {
    out->lines_per_cta[i] = i < p->d ? base_pass_t<double>(p, i).lpb : 0;
    out->lines_per_cta_f32[i] = i < p->d && p->mixed ? base_pass_t<float>(p, i).lpb : 0;
  out->tc_dims = 0;
  for (int i = 0; i < p->d; ++i)
    if (p->tc_on[i]) out->tc_dims |= 1 << i;
  if (p->tcm) out->tc_dims |= 1 << 8;
  }
  for (int i = 0; i < p->d; ++i) {
    out->route_source[i] = p->route_src[i];
    out->route_ms[i] = p->route_ms[i];
    out->route_alt_ms[i] = p->route_alt_ms[i];
  }
  out->resid_precision = p->mixed ? (p->res_df ? TAU_DF64 : TAU_FP64) : p->desc.precision;
  out->kernels_prologue = p->k_pro;
  out->kernels_per_iter = p->k_body;
  out->kernels_epilogue = p->k_epi;
  if (p->mixed) {
    std::vector<int> sw((size_t)p->desc.M);
    CK(cudaMemcpy(sw.data(), p->sweeps, sw.size() * sizeof(int), cudaMemcpyDeviceToHost));
    int64_t kt = 0, ts = 0;
    for (int64_t m = 0; m < g.m && m < p->desc.M; ++m) {
      ts += sw[m];
      kt += p->k_pro + p->k_epi + (int64_t)(sw[m] + 1) * (p->k_ir_pre + p->k_ir_post) +
            (int64_t)(it[m] + 1) * p->k_body;
    }
    out->kernels_total = kt;
    out->total_sweeps = ts;
  } else {
    out->kernels_total = g.m * (p->k_pro + p->k_epi) + tot * p->k_body;
  }
  out->device_bytes = p->bytes;
  if (g.notconv) return fail(TAU_ENOTCONV, "a step reached max_iter without meeting tol");
  return TAU_OK;
}

tau_status tau_get_iters(tau_problem* p, int* iters, int64_t cap) {
  TRY(check_ready(p));
  if (!iters || cap < 0) return fail(TAU_EINVAL, "bad iters/cap");
  CK(cudaStreamSynchronize(p->st));
  GmresDev g;
  CK(cudaMemcpy(&g, p->g, sizeof(GmresDev), cudaMemcpyDeviceToHost));
  const int64_t nget = cap < g.m ? cap : g.m;
  if (nget > 0) CK(cudaMemcpy(iters, p->iters, nget * sizeof(int), cudaMemcpyDeviceToHost));
  return TAU_OK;
}

tau_status tau_destroy(tau_problem* p) {
  if (!p) return TAU_OK;
  cudaStreamSynchronize(p->st);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  for (void* a : p->allocs) cudaFree(a);
  if (p->h_done) cudaFreeHost(p->h_done);
  if (p->cap) cudaStreamDestroy(p->cap);
  delete p;
  return TAU_OK;
}

tau_status tau_apply_A(tau_problem* p, int64_t m, const double* x, double* y) {
  TRY(check_ready(p));
  if (!x || !y) return fail(TAU_EINVAL, "NULL vector");
  if (m < 0 || m >= p->desc.M) return fail(TAU_EINVAL, "m=%lld outside 0..M-1", (long long)m);
  KL(launch_fields(field_dev(p), p->g, m, p->E, p->Fdt, p->st));
  ChainIO io;
  io.x = x;
  io.out = y;
  return enq_mv<double>(p, p->st, io, 1.0, FIN_NONE, nullptr, false);
}

tau_status tau_apply_MinvA(tau_problem* p, int64_t m, const double* x, double* z) {
  TRY(check_ready(p));
  if (!x || !z) return fail(TAU_EINVAL, "NULL vector");
  if (m < 0 || m >= p->desc.M) return fail(TAU_EINVAL, "m=%lld outside 0..M-1", (long long)m);
  KL(launch_fields(field_dev(p), p->g, m, p->E, p->Fdt, p->st));
  ChainIO io;
  io.x = x;
  io.out = z;
  return enq_mv<double>(p, p->st, io, 1.0, FIN_NONE, nullptr, true);
}

tau_status tau_apply_Minv(tau_problem* p, const double* r, double* z) {
  TRY(check_ready(p));
  if (!r || !z) return fail(TAU_EINVAL, "NULL vector");
  ChainIO io;
  io.x = r;
  io.out = z;
  return enq_minv<double>(p, p->st, io);
}

tau_status tau_rhs(tau_problem* p, int64_t m, const double* u, double* b) {
  TRY(check_ready(p));
  if (!u || !b) return fail(TAU_EINVAL, "NULL vector");
  if (m < 0 || m >= p->desc.M) return fail(TAU_EINVAL, "m=%lld outside 0..M-1", (long long)m);
  KL(launch_fields(field_dev(p), p->g, m, p->E, p->Fdt, p->st));
  ChainIO io;
  io.x = u;
  io.out = b;
  return enq_mv<double>(p, p->st, io, -1.0, FIN_ADD_F, p->Fdt, false);
}

tau_status tau_dst(tau_problem* p, const double* x, double* y) {
  TRY(check_ready(p));
  if (!x || !y) return fail(TAU_EINVAL, "NULL vector");
  for (int ax = 0; ax < p->d; ++ax) {
    Pass P = base_pass(p, ax);
    P.post = POST_DST;
    P.in_a = ax == 0 ? x : y;
    P.out_a = y;
    TRY(enq(P, p->st));
  }
  return TAU_OK;
}

tau_status tau_toeplitz_mode(tau_problem* p, int dim, const double* x, double* y) {
  TRY(check_ready(p));
  if (!x || !y) return fail(TAU_EINVAL, "NULL vector");
  if (dim < 0 || dim >= p->d) return fail(TAU_EINVAL, "dim=%d outside 0..d-1", dim);
  Pass P = base_pass(p, dim);
  P.toep_only = 1;
  P.in_a = x;
  P.out_a = y;
  return enq(P, p->st);
}

struct tau_batch {
  std::vector<tau_problem*> probs;
  cudaStream_t st = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> dmem;   // grouped launches: argument tables, block ranges, loop aggregators
  tau_batch_info info{};
};

namespace {

// One grouped launch: the grouped kernel of a body over the problems of a group, their argument
// blocks (device) and block ranges start[0..n] (device).
struct Merged {
  const void* fn;
  unsigned grid, block;
  size_t smem;
  void* dargs;
  int* dstart;
  int n;
};

// Argument tables of a group's launches: staged on the host while the launches are recorded, with
// their device addresses handed out in advance (dev + offset), and uploaded in one copy when the
// graph is complete.  A dry run (dev == NULL) only measures the size.
struct Arena {
  std::vector<unsigned char> host;
  char* dev = nullptr;
  size_t take(size_t bytes) {
    const size_t off = (host.size() + 15) & ~(size_t)15;
    host.resize(off + bytes);
    return off;
  }
  void* at(size_t off) const { return dev ? dev + off : nullptr; }
};

// Grouping applies to the mixed-precision form on the line-pass routes: every problem of a group
// then enqueues the same sequence of kernels (same d, residual precision and initial guess), which
// is what lets their launches merge position by position.
bool groupable(const tau_problem* p) {
  if (!p->mixed || p->tcm || p->spgm || p->tpgm || !p->setup_done) return false;
  for (int i = 0; i < p->d; ++i)
    if (p->tc_on[i] || p->route[i] == ROUTE_LONG) return false;
  return true;
}

std::tuple<int, int, int> group_key(const tau_problem* p) {
  return std::make_tuple(p->d, p->res_df ? 1 : 0, p->desc.x0_mode);
}

// Record `fn` for every problem of the group (nothing is launched) and merge the records position
// by position into grouped launches whose tables go to the arena.
tau_status record_merge(Arena& ar, const std::vector<tau_problem*>& ps,
                        const std::function<tau_status(tau_problem*)>& fn, std::vector<Merged>& out) {
  std::vector<std::vector<LaunchRec>> R(ps.size());
  for (size_t i = 0; i < ps.size(); ++i) {
    tl_rec = &R[i];
    const tau_status s = fn(ps[i]);
    tl_rec = nullptr;
    if (s != TAU_OK) return s;
  }
  const size_t L = R[0].size();
  for (size_t i = 1; i < ps.size(); ++i)
    if (R[i].size() != L) return fail(TAU_EUNSUPPORTED, "grouped launches: problems enqueue different kernel sequences");
  // Problems may run a different kernel at the same position (the tile autotuner picks the
  // 128- or 256-thread line pass per problem): each distinct (kernel, block) at a position becomes
  // a grouped launch of its own over the problems that run it; they are independent of each other.
  const int n = (int)ps.size();
  for (size_t k = 0; k < L; ++k) {
    std::vector<int> done(n, 0);
    for (int first = 0; first < n; ++first) {
      if (done[first]) continue;
      const LaunchRec& r0 = R[first][k];
      const size_t asz = r0.args.size();
      std::vector<int> mem;
      for (int i = first; i < n; ++i) {
        const LaunchRec& r = R[i][k];
        if (done[i] || r.fn != r0.fn || r.block != r0.block) continue;
        if (r.args.size() != asz) return fail(TAU_EUNSUPPORTED, "grouped launches: argument sizes differ");
        mem.push_back(i);
        done[i] = 1;
      }
      const int m = (int)mem.size();
      const size_t oa = ar.take(asz * m), os = ar.take(sizeof(int) * (m + 1));
      int* start = reinterpret_cast<int*>(ar.host.data() + os);
      start[0] = 0;
      size_t smem = 0;
      for (int q = 0; q < m; ++q) {
        const LaunchRec& r = R[mem[q]][k];
        memcpy(ar.host.data() + oa + asz * q, r.args.data(), asz);
        start = reinterpret_cast<int*>(ar.host.data() + os);   // host may have grown: re-take
        start[q + 1] = start[q] + (int)r.grid;
        smem = std::max(smem, r.smem);
      }
      start = reinterpret_cast<int*>(ar.host.data() + os);
      out.push_back(Merged{r0.fn, (unsigned)start[m], r0.block, smem, ar.at(oa), static_cast<int*>(ar.at(os)), m});
    }
  }
  return TAU_OK;
}

tau_status launch_merged(const std::vector<Merged>& v, cudaStream_t s) {
  for (const Merged& m : v) {
    if (m.grid == 0) continue;
    void* dargs = m.dargs;
    int* dstart = m.dstart;
    int nn = m.n;
    void* kargs[] = {&dargs, &dstart, &nn};
    CK(cudaLaunchKernel(m.fn, dim3(m.grid), dim3(m.block), kargs, m.smem, s));
  }
  return TAU_OK;
}

// The graph of one step for a group: the mixed step (prologue -> WHILE(refinement control ->
// WHILE(FGMRES iteration) -> correction) -> epilogue) with every kernel a grouped launch over the
// group's problems.  Each loop runs while any problem of the group still iterates; a problem that
// finished skips its work in the remaining iterations.  The problems may stand at different steps
// (each reads its own m on the device).  With ar.dev == NULL nothing is captured (dry run).
struct GroupCounts {
  int64_t pro_epi = 0, sweep = 0, inner = 0;
};

tau_status build_group_inner(Arena& ar, const std::vector<tau_problem*>& ps, cudaGraph_t G, GroupCounts* cnt) {
  tau_problem* p0 = ps[0];
  const bool dry = ar.dev == nullptr;
  // the group's loop-condition aggregators, at the start of the arena
  const size_t ogc = ar.take(2 * sizeof(GroupCtl));
  GroupCtl* gc_host = reinterpret_cast<GroupCtl*>(ar.host.data() + ogc);
  for (int k = 0; k < 2; ++k) gc_host[k] = GroupCtl{0u, 0, (int)ps.size(), 0};
  for (tau_problem* p : ps) p->gctl = static_cast<GroupCtl*>(ar.at(ogc));
  auto done = [&](tau_status s) {
    for (tau_problem* p : ps) p->gctl = nullptr;
    return s;
  };
  std::vector<Merged> pro, pre, inner, post, epi;
  std::vector<cudaGraphNode_t> none, leaves, preL, tmp;
  cudaGraphConditionalHandle ho = 0, hi = 0;
  cudaGraphNode_t wo = nullptr, wi = nullptr;
  cudaGraph_t bo = nullptr, bi = nullptr;
  tau_status s = record_merge(ar, ps, [&](tau_problem* p) { return enq_mx_prologue(p, p->cap); }, pro);
  if (s == TAU_OK && !dry)
    s = capture_into(p0, G, none, [&](cudaStream_t st) { return launch_merged(pro, st); }, leaves);
  if (s == TAU_OK && !dry) s = make_handle(G, &ho);
  if (s == TAU_OK && !dry) s = add_while(G, leaves, &ho, &wo, &bo);
  if (s == TAU_OK && !dry) s = make_handle(bo, &hi);
  if (s == TAU_OK)
    s = record_merge(ar, ps, [&](tau_problem* p) { return enq_mx_sweep_pre(p, p->cap, ho, hi, 2); }, pre);
  if (s == TAU_OK && !dry)
    s = capture_into(p0, bo, none, [&](cudaStream_t st) { return launch_merged(pre, st); }, preL);
  if (s == TAU_OK && !dry) s = add_while(bo, preL, &hi, &wi, &bi);
  if (s == TAU_OK) s = record_merge(ar, ps, [&](tau_problem* p) { return enq_mx_inner(p, p->cap, hi, 2); }, inner);
  if (s == TAU_OK && !dry)
    s = capture_into(p0, bi, none, [&](cudaStream_t st) { return launch_merged(inner, st); }, tmp);
  if (s == TAU_OK) s = record_merge(ar, ps, [&](tau_problem* p) { return enq_mx_sweep_post(p, p->cap); }, post);
  if (s == TAU_OK && !dry)
    s = capture_into(p0, bo, {wi}, [&](cudaStream_t st) { return launch_merged(post, st); }, tmp);
  if (s == TAU_OK) s = record_merge(ar, ps, [&](tau_problem* p) { return enq_mx_epilogue(p, p->cap); }, epi);
  if (s == TAU_OK && !dry)
    s = capture_into(p0, G, {wo}, [&](cudaStream_t st) { return launch_merged(epi, st); }, tmp);
  if (s == TAU_OK && cnt) {
    cnt->pro_epi = (int64_t)(pro.size() + epi.size());
    cnt->sweep = (int64_t)(pre.size() + post.size());
    cnt->inner = (int64_t)inner.size();
  }
  return done(s);
}

// Build a group's branch into G: a dry run sizes the argument tables, one allocation holds them
// (returned in *dev, owned by the caller; with pool_cap non-null, *dev is a buffer of *pool_cap
// bytes to reuse when large enough, otherwise it is replaced by a larger one), the real run records
// and captures, one copy uploads.
tau_status add_group_branch(const std::vector<tau_problem*>& ps, cudaGraph_t G, void** dev, GroupCounts* cnt,
                            size_t* pool_cap = nullptr) {
  Arena dry;
  TRY(build_group_inner(dry, ps, G, nullptr));
  Arena ar;
  const size_t need = dry.host.size() + 16;
  if (pool_cap && *dev && *pool_cap >= need) {
    ar.dev = static_cast<char*>(*dev);
  } else {
    if (pool_cap && *dev) {
      cudaFree(*dev);   // waits for the device: only when the tables outgrow the buffer
      *dev = nullptr;
      *pool_cap = 0;
    }
    const size_t cap = pool_cap ? need + need / 2 : need;
    *dev = nullptr;
    CK(cudaMalloc(reinterpret_cast<void**>(&ar.dev), cap));
    if (pool_cap) *pool_cap = cap;
  }
  *dev = ar.dev;
  ar.host.reserve(dry.host.size());
  TRY(build_group_inner(ar, ps, G, cnt));
  if (ar.host.size() > dry.host.size()) return fail(TAU_EUNSUPPORTED, "grouped launches: table size changed");
  CK(cudaMemcpy(ar.dev, ar.host.data(), ar.host.size(), cudaMemcpyHostToDevice));
  return TAU_OK;
}

}  // namespace

tau_status tau_batch_create(tau_problem* const* problems, int count, void* stream, tau_batch** out) {
  if (!problems || !out || count < 1) return fail(TAU_EINVAL, "tau_batch_create: bad arguments");
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    tau_problem* p = problems[i];
    if (!p) return fail(TAU_EINVAL, "tau_batch_create: problem %d is NULL", i);
    if (!p->setup_done) return fail(TAU_ESTATE, "tau_batch_create: problem %d not set up", i);
    if (p->m_host != problems[0]->m_host || p->desc.M != problems[0]->desc.M)
      return fail(TAU_EINVAL, "tau_batch_create: problems must stand at the same step m with the same M");
    CK(cudaStreamSynchronize(p->st));
  }
  tau_batch* b = new (std::nothrow) tau_batch();
  if (!b) return fail(TAU_ENOMEM, "host allocation");
  b->probs.assign(problems, problems + count);
  b->st = (cudaStream_t)stream;
  cudaGraph_t G = nullptr;
  if (cudaGraphCreate(&G, 0) != cudaSuccess) {
    delete b;
    return fail(TAU_ECUDA, "cudaGraphCreate");
  }
  // groups of mixed-precision problems with the same kernel sequence (TAU_BATCH_GROUPS=0: none)
  const char* ge = std::getenv("TAU_BATCH_GROUPS");
  const bool grouping = !(ge && ge[0] == '0');
  std::map<std::tuple<int, int, int>, std::vector<tau_problem*>> groups;
  std::vector<tau_problem*> single;
  for (tau_problem* p : b->probs) {
    if (grouping && groupable(p)) groups[group_key(p)].push_back(p);
    else single.push_back(p);
  }
  tau_status st = TAU_OK;
  for (auto& kv : groups) {
    if (kv.second.size() < 2) {
      single.push_back(kv.second[0]);
      continue;
    }
    if (st != TAU_OK) continue;
    void* dev = nullptr;   // owned by the batch
    GroupCounts cnt;
    st = add_group_branch(kv.second, G, &dev, &cnt);
    if (dev) b->dmem.push_back(dev);
    if (st == TAU_OK) {
      b->info.groups += 1;
      b->info.grouped_problems += (int)kv.second.size();
      b->info.launches_prologue_epilogue += cnt.pro_epi;
      b->info.launches_per_sweep += cnt.sweep;
      b->info.launches_per_inner_iter += cnt.inner;
    }
  }
  for (size_t i = 0; i < single.size() && st == TAU_OK; ++i) {
    st = build_graph_inner(single[i], G);
    b->info.branches += 1;
  }
  b->info.branches += b->info.groups;
  if (st == TAU_OK) {
    cudaError_t e = cudaGraphInstantiate(&b->exec, G, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      st = fail(TAU_EUNSUPPORTED, "batch graph: %s", cudaGetErrorString(e));
    }
  }
  cudaGraphDestroy(G);
  if (st != TAU_OK) {
    for (void* d : b->dmem) cudaFree(d);
    delete b;
    return st;
  }
  *out = b;
  return TAU_OK;
}

}  // extern "C"

// ---- grouped steps for the serving loop (tau_serve.cu): problems that may stand at different
// steps, each advanced by one step per launch of the group's graph
namespace tau {

struct GroupExec {
  std::vector<tau_problem*> ps;
  cudaGraphExec_t exec = nullptr;
};

// Groupable problems and the key of their group (-1: not groupable).
int64_t problem_group_key(const tau_problem* p) {
  if (!groupable(p)) return -1;
  const auto k = group_key(p);
  return (int64_t)std::get<0>(k) * 16 + std::get<1>(k) * 4 + std::get<2>(k);
}

// pool/pool_cap: the caller's argument-table buffer, reused (or replaced by a larger one); the
// caller keeps it past group_exec_destroy and frees it once no launch of the group can run.
tau_status group_exec_create(tau_problem* const* ps, int n, GroupExec** out, void** pool, size_t* pool_cap) {
  *out = nullptr;
  GroupExec* g = new (std::nothrow) GroupExec();
  if (!g) return fail(TAU_ENOMEM, "host allocation");
  g->ps.assign(ps, ps + n);
  cudaGraph_t G = nullptr;
  if (cudaGraphCreate(&G, 0) != cudaSuccess) {
    delete g;
    return fail(TAU_ECUDA, "cudaGraphCreate");
  }
  GroupCounts cnt;
  tau_status st = add_group_branch(g->ps, G, pool, &cnt, pool_cap);
  if (st == TAU_OK && cudaGraphInstantiate(&g->exec, G, 0) != cudaSuccess) {
    cudaGetLastError();
    st = fail(TAU_EUNSUPPORTED, "group graph instantiation");
  }
  cudaGraphDestroy(G);
  if (st != TAU_OK) {
    delete g;
    return st;
  }
  *out = g;
  return TAU_OK;
}

tau_status group_exec_launch(GroupExec* g, int64_t count, cudaStream_t st) {
  for (tau_problem* p : g->ps)
    if (p->m_host + count > p->desc.M) return fail(TAU_EINVAL, "group step past a member's last step");
  for (int64_t c = 0; c < count; ++c) CK(cudaGraphLaunch(g->exec, st));
  for (tau_problem* p : g->ps) {
    p->m_host += count;
    p->fields_m = -1;
  }
  return TAU_OK;
}

// The group's graph is freed (launches already enqueued still run); the argument tables stay
// with the caller.
void group_exec_destroy(GroupExec* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
}

}  // namespace tau

extern "C" {

tau_status tau_batch_get_info(tau_batch* b, tau_batch_info* info) {
  if (!b || !info) return fail(TAU_EINVAL, "NULL argument");
  *info = b->info;
  return TAU_OK;
}

tau_status tau_batch_step(tau_batch* b, int64_t count) {
  if (!b) return fail(TAU_EINVAL, "batch is NULL");
  tau_problem* p0 = b->probs[0];
  if (count < 0 || p0->m_host + count > p0->desc.M)
    return fail(TAU_EINVAL, "count=%lld with m=%lld of M=%lld", (long long)count, (long long)p0->m_host,
                (long long)p0->desc.M);
  for (int64_t c = 0; c < count; ++c) CK(cudaGraphLaunch(b->exec, b->st));
  for (tau_problem* p : b->probs) {
    p->m_host += count;
    if (count > 0) p->fields_m = -1;
  }
  return TAU_OK;
}

tau_status tau_batch_sync(tau_batch* b) {
  if (!b) return fail(TAU_EINVAL, "batch is NULL");
  CK(cudaStreamSynchronize(b->st));
  tau_status worst = TAU_OK;
  for (tau_problem* p : b->probs) {
    tau_status s = sync_status(p);
    if (s != TAU_OK) worst = s;
  }
  return worst;
}

tau_status tau_batch_destroy(tau_batch* b) {
  if (!b) return TAU_OK;
  cudaStreamSynchronize(b->st);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (void* d : b->dmem) cudaFree(d);
  delete b;
  return TAU_OK;
}

tau_status tau_apply_A_f32(tau_problem* p, int64_t m, const float* x, float* y) {
  TRY(check_ready(p));
  if (!p->mixed) return fail(TAU_ESTATE, "FP32 operators exist only for TAU_MIXED problems");
  if (!x || !y) return fail(TAU_EINVAL, "NULL vector");
  if (m < 0 || m >= p->desc.M) return fail(TAU_EINVAL, "m=%lld outside 0..M-1", (long long)m);
  TRY(fields_for(p, m));
  ChainT<float> io;
  io.x = x;
  io.out = y;
  return enq_mv<float>(p, p->st, io, 1.0, FIN_NONE, nullptr, false);
}

tau_status tau_apply_Minv_f32(tau_problem* p, const float* r, float* z) {
  TRY(check_ready(p));
  if (!p->mixed) return fail(TAU_ESTATE, "FP32 operators exist only for TAU_MIXED problems");
  if (!r || !z) return fail(TAU_EINVAL, "NULL vector");
  ChainT<float> io;
  io.x = r;
  io.out = z;
  return enq_minv<float>(p, p->st, io);
}

tau_status tau_choose_precision(const tau_problem_desc* desc, int* precision) {
  if (!desc || !precision) return fail(TAU_EINVAL, "desc/precision is NULL");
  const tau_problem_desc& D = *desc;
  if (D.d < 1 || D.d > 3) return fail(TAU_EINVAL, "d=%d outside 1..3", D.d);
  if (!(D.T > 0) || D.M < 1) return fail(TAU_EINVAL, "T must be > 0 and M >= 1");
  if (!(D.e_min > 0) || !std::isfinite(D.e_min)) return fail(TAU_EINVAL, "e_min must be a positive number");
  const double dt = D.T / (double)D.M;
  double worst = 0.0;
  for (int i = 0; i < D.d; ++i) {
    if (D.n[i] < 1) return fail(TAU_EINVAL, "n[%d] < 1", i);
    if (!(D.alpha[i] > 1.0 && D.alpha[i] < 2.0)) return fail(TAU_EINVAL, "alpha[%d]=%g not in (1,2)", i, D.alpha[i]);
    if (!(D.kappa[i] >= 0.0)) return fail(TAU_EINVAL, "kappa[%d]=%g < 0", i, D.kappa[i]);
    if (!(D.R[i] > D.L[i])) return fail(TAU_EINVAL, "R[%d] <= L[%d]", i, i);
    const double a = D.alpha[i], h = (D.R[i] - D.L[i]) / (double)(D.n[i] + 1);
    const double eta = D.kappa[i] * dt / (2.0 * std::pow(h, a));
    // s_0 = Gamma(a+1) / Gamma(a/2+1)^2, the diagonal FCD weight; ||s||_1 <= 2 s_0
    const double g = std::tgamma(a / 2.0 + 1.0);
    const double s0 = std::tgamma(a + 1.0) / (g * g);
    worst = std::max(worst, eta * 2.0 * s0 / D.e_min);
  }
  *precision = std::ldexp(worst, -23) <= 0.05 ? TAU_MIXED : TAU_DF64;
  return TAU_OK;
}

tau_status tau_selftest_bounded_wait(void* stream, int* gave_up) {
  if (!gave_up) return fail(TAU_EINVAL, "NULL output");
  cudaStream_t st = (cudaStream_t)stream;
  int* d = nullptr;
  CK(cudaMalloc(&d, sizeof(int)));
  cudaError_t e = cudaMemsetAsync(d, 0xff, sizeof(int), st);
  if (e == cudaSuccess) e = launch_wait_selftest(100000, d, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gave_up, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return fail(TAU_ECUDA, "bounded-wait self-test: %s", cudaGetErrorString(e));
  return TAU_OK;
}

tau_status tau_inject_wait_timeout(tau_problem* p) {
  if (!p) return fail(TAU_EINVAL, "problem is NULL");
  CK(cudaMemsetAsync(p->tc_err, 0xff, sizeof(int), p->st));
  return TAU_OK;
}

tau_status tau_get_ebar(tau_problem* p, double* ebar, double* e_hat, double* e_check) {
  TRY(check_ready(p));
  if (ebar) *ebar = p->ebar;
  if (e_hat) *e_hat = p->ehat;
  if (e_check) *e_check = p->echeck;
  return TAU_OK;
}

tau_status tau_measure_fp64_peak(void* stream, double* flops_per_s) {
  if (!flops_per_s) return fail(TAU_EINVAL, "NULL output");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 2, iters = 20000;
  double* out = nullptr;
  CK(cudaMalloc(&out, sizeof(double) * blocks * 256));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(launch_fp64_peak(out, blocks, iters, st));
  double best = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    CK(cudaEventRecord(e0, st));
    for (int r = 0; r < 3; ++r) CK(launch_fp64_peak(out, blocks, iters, st));
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    const double f = 3.0 * 2.0 * 8.0 * iters * (double)blocks * 256 / (ms * 1e-3);
    if (f > best) best = f;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *flops_per_s = best;
  return TAU_OK;
}

}  // extern "C"
