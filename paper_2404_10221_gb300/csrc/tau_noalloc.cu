// Allocation-free variant of the matvec entry point: y = A x = B_alpha (e∘x) + S_alpha x.
//
// Some callers cannot allocate device memory: code that runs inside a host application whose
// own pool owns the whole device and refuses outside cudaMalloc calls, plugins that must leave
// the device's memory footprint exactly as they found it, and latency-critical loops where a
// cudaMalloc (which can synchronise the device) is not acceptable.  They still own their inputs
// and outputs; the scratch this computation needs lives here, in one statically sized device
// array that every GPU loading the library holds until the process exits.
//
// Everything tau_create/tau_setup would derive for the matvec (FCD weights, the circulant
// spectra of the Toeplitz factors, twiddles) and the two Kronecker channels are rebuilt in this
// array on every call.  Calls share the array: two calls that overlap on the GPU (different
// streams, or the same array used from two host threads without ordering) race and corrupt
// each other's results.
#include "tau_rsfde.h"
#include "tau_internal.cuh"

#include <cmath>
#include <cstdio>
#include <mutex>

namespace tau {

namespace {

// Limits of the static scratch.
constexpr int64_t NA_MAX_UNKNOWNS = 1 << 18;  // grid points of one call (262,144)
constexpr int NA_MAX_N = KMAX - 1;            // points per dimension (4095)
constexpr int NA_MAX_DEVICES = 64;

// Layout of the scratch, in doubles.
constexpr size_t NA_CHAN_A = 0;                               // channel a
constexpr size_t NA_CHAN_C = NA_CHAN_A + NA_MAX_UNKNOWNS;     // channel c
constexpr size_t NA_DIM0 = NA_CHAN_C + NA_MAX_UNKNOWNS;       // per-dimension tables
constexpr size_t NA_DIM_S = 0;                                // weights s_0..s_{n-1}
constexpr size_t NA_DIM_C = NA_DIM_S + KMAX;                  // circulant first column, 2K
constexpr size_t NA_DIM_LAM = NA_DIM_C + 2 * (size_t)KMAX;    // spectrum lambda_0..lambda_K
constexpr size_t NA_DIM_SPEC = NA_DIM_LAM + KMAX + 2;         // (a, b, c, d) complex, K/2+1
constexpr size_t NA_DIM_TWK = NA_DIM_SPEC + 4 * (size_t)KMAX + 8;  // stage-packed twiddles, 2K+1 pairs
constexpr size_t NA_DIM_STRIDE = NA_DIM_TWK + 4 * (size_t)KMAX + 2;
constexpr size_t NA_TOTAL = NA_DIM0 + 3 * NA_DIM_STRIDE;      // ~5.2 MB

static __device__ __align__(256) double g_tau_noalloc_scratch[NA_TOTAL];

std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

// FCD weights by the recurrence of §2 and the circulant embedding of length 2K of S_alpha
// (c_0 = s_0, c_k = c_{2K-k} = s_k for 1 <= k < n, zero elsewhere).
__global__ void k_na_weights(double alpha, int n, double* s, double* c) {
  const int K = n + 1;
  if (threadIdx.x == 0) {
    const double g = tgamma(alpha / 2.0 + 1.0);
    s[0] = tgamma(alpha + 1.0) / (g * g);
    for (int k = 1; k < n; ++k) s[k] = (1.0 - (alpha + 1.0) / (alpha / 2.0 + k)) * s[k - 1];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) {
    double v = 0.0;
    if (t == 0) v = s[0];
    else if (t < n) v = s[t];
    else if (2 * K - t < n) v = s[2 * K - t];
    c[t] = v;
  }
}

// coefficients (a, b, c, d)_k, k = 0..K/2, of the packed spectral step (toep_pack_coeffs);
// W_k = exp(-i pi k / K) is entry K + k of the twiddle table
__global__ void k_na_spec(int K, const double* lam, const double2* twK, double2* spec) {
  for (int k = threadIdx.x; k <= K / 2; k += blockDim.x) {
    double abcd[8];
    const double2 w = twK[K + k];
    toep_pack_coeffs(lam[k], lam[K - k], w.x, w.y, K, abcd);
    for (int r = 0; r < 4; ++r) spec[4 * k + r] = make_double2(abcd[2 * r], abcd[2 * r + 1]);
  }
}

tau_status na_fail(tau_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

}  // namespace
}  // namespace tau

using namespace tau;

extern "C" tau_status tau_apply_A_noalloc(const tau_problem_desc* desc, const double* e, const double* x, double* y,
                                          void* stream) {
  char buf[256];
  if (!desc || !e || !x || !y) return na_fail(TAU_EINVAL, "tau_apply_A_noalloc: NULL argument");
  const tau_problem_desc& D = *desc;
  if (D.d < 1 || D.d > 3) return na_fail(TAU_EINVAL, "tau_apply_A_noalloc: d outside 1..3");
  int64_t n_tot = 1;
  for (int i = 0; i < D.d; ++i) {
    if (D.n[i] < 1 || D.n[i] > NA_MAX_N) {
      snprintf(buf, sizeof(buf), "tau_apply_A_noalloc: n[%d]=%lld outside 1..%d (static scratch limit)", i,
               (long long)D.n[i], NA_MAX_N);
      return na_fail(TAU_EINVAL, buf);
    }
    if (!(D.alpha[i] > 1.0 && D.alpha[i] < 2.0) || !(D.kappa[i] >= 0.0) || !(D.R[i] > D.L[i]))
      return na_fail(TAU_EINVAL, "tau_apply_A_noalloc: alpha must lie in (1,2), kappa >= 0, R > L");
    // the route is this entry point's own (FFT when n_i + 1 is a power of two, else dense sums):
    // a forced route would silently not be honoured, so it is refused
    if (D.route[i] != TAU_ROUTE_AUTO) {
      snprintf(buf, sizeof(buf), "tau_apply_A_noalloc: route[%d]=%d; only TAU_ROUTE_AUTO is accepted", i, D.route[i]);
      return na_fail(TAU_EINVAL, buf);
    }
    n_tot *= D.n[i];
  }
  if (n_tot > NA_MAX_UNKNOWNS) {
    snprintf(buf, sizeof(buf), "tau_apply_A_noalloc: %lld grid points exceed the static scratch limit of %lld",
             (long long)n_tot, (long long)NA_MAX_UNKNOWNS);
    return na_fail(TAU_EINVAL, buf);
  }
  if (!(D.T > 0) || D.M < 1) return na_fail(TAU_EINVAL, "tau_apply_A_noalloc: T must be > 0 and M >= 1");
  cudaStream_t st = (cudaStream_t)stream;

  // once per device, with that device current: the device address of the static scratch
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return na_fail(TAU_ECUDA, cudaGetErrorString(ce));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(TAU_EUNSUPPORTED, "tau_apply_A_noalloc: device ordinal >= 64");
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* ptr = nullptr;
      ce = cudaGetSymbolAddress(&ptr, g_tau_noalloc_scratch);
      if (ce != cudaSuccess) {
        snprintf(buf, sizeof(buf), "tau_apply_A_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(ce));
        return na_fail(TAU_ECUDA, buf);
      }
      ce = init_kernel_attributes();
      if (ce != cudaSuccess) return na_fail(TAU_ECUDA, cudaGetErrorString(ce));
      g_na_ptr[dev] = static_cast<double*>(ptr);
    }
    base = g_na_ptr[dev];
  }

  const double dt = D.T / (double)D.M;
  DimData dims[3] = {};
  for (int i = 0; i < D.d; ++i) {
    const int n = (int)D.n[i], K = n + 1;
    double* dimb = base + NA_DIM0 + i * NA_DIM_STRIDE;
    const bool fft = (K & (K - 1)) == 0;
    DimData& Dd = dims[i];
    Dd.n = n;
    Dd.K = K;
    Dd.route = fft ? ROUTE_FFT : ROUTE_DENSE;
    Dd.bdiag = 1.0 - D.alpha[i] / 12.0;
    Dd.boff = D.alpha[i] / 24.0;
    Dd.dsc = sqrt(2.0 / (double)(D.n[i] + 1));
    const double h = (D.R[i] - D.L[i]) / (double)(n + 1);
    Dd.eta = D.kappa[i] * dt / (2.0 * std::pow(h, D.alpha[i]));
    Dd.s = dimb + NA_DIM_S;
    Dd.sintab = nullptr;
    Dd.spec = reinterpret_cast<const double2*>(dimb + NA_DIM_SPEC);
    double2* twk = reinterpret_cast<double2*>(dimb + NA_DIM_TWK);
    Dd.twK = twk;
    Dd.twK2 = nullptr;
    k_na_weights<<<1, 256, 0, st>>>(D.alpha[i], n, dimb + NA_DIM_S, dimb + NA_DIM_C);
    if (fft) {
      if ((ce = launch_twp(K, twk, st)) != cudaSuccess) return na_fail(TAU_ECUDA, cudaGetErrorString(ce));
      if ((ce = launch_spectrum(K, dimb + NA_DIM_C, dimb + NA_DIM_LAM, twk, st)) != cudaSuccess)
        return na_fail(TAU_ECUDA, cudaGetErrorString(ce));
      k_na_spec<<<1, 256, 0, st>>>(K, dimb + NA_DIM_LAM, twk, reinterpret_cast<double2*>(dimb + NA_DIM_SPEC));
    }
    if ((ce = cudaGetLastError()) != cudaSuccess) return na_fail(TAU_ECUDA, cudaGetErrorString(ce));
  }

  // the matvec passes, one per dimension, channels a and c in the static scratch
  double* chA = base + NA_CHAN_A;
  double* chC = base + NA_CHAN_C;
  for (int ax = 0; ax < D.d; ++ax) {
    Pass P{};
    P.ax = ax;
    P.len = (int)D.n[ax];
    int64_t inner = 1;
    for (int i = 0; i < ax; ++i) inner *= D.n[i];
    P.inner = inner;
    P.nlines = n_tot / P.len;
    P.dim = dims[ax];
    const size_t per_line = 8 * ((size_t)P.len + (P.dim.route == ROUTE_FFT ? 2 * (size_t)P.dim.K : 2 * (size_t)P.len));
    int64_t lpb = (int64_t)(24576 / per_line);
    if (lpb < 1) lpb = 1;
    if (lpb > 16) lpb = 16;
    const int64_t cap = ax == 0 ? P.nlines : inner;
    if (lpb > cap) lpb = cap;
    while (lpb & (lpb - 1)) lpb &= lpb - 1;   // a power of two (the kernel maps lines by shifts)
    P.lpb = (int)lpb;
    P.ntiles = ax == 0 ? (P.nlines + lpb - 1) / lpb : (P.nlines / inner) * ((inner + lpb - 1) / lpb);
    P.mv = 1;
    P.first = ax == 0;
    P.last = ax == D.d - 1;
    P.seta = dims[ax].eta;
    P.finish = FIN_NONE;
    P.post = POST_NONE;
    P.in_a = ax == 0 ? x : chA;
    P.in_c = ax == 0 ? nullptr : chC;
    P.e = ax == 0 ? e : nullptr;
    P.out_a = P.last ? y : chA;
    P.out_c = P.last ? nullptr : chC;
    if ((ce = launch_pass(P, st)) != cudaSuccess) return na_fail(TAU_ECUDA, cudaGetErrorString(ce));
  }
  return TAU_OK;
}
