// Internal declarations of the τ-GMRES CUDA library (device helpers, pass
// descriptors, host launchers).  Not part of the public C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace tau {

// Virtual block of a kernel body (tau_group.cuh): (blockIdx.x, gridDim.x) in a plain launch; the
// block's index and count within its problem's range in a grouped launch.
struct VB {
  int bid, nb;
};

// Aggregation of one device-controlled loop condition over the n problems of a group.
struct GroupCtl {
  unsigned int ticket;
  int any;
  int n;
  int pad;
};

// A recorded launch: the grouped kernel of the body, its argument bytes, grid, block, shared memory.
struct LaunchRec {
  const void* fn;
  std::vector<unsigned char> args;
  unsigned grid, block;
  size_t smem;
  int kthreads;
};
// When set, the launch functions of the mixed-precision step record instead of launching.
extern thread_local std::vector<LaunchRec>* tl_rec;

// Largest half-length complex FFT size K = n + 1 of the FFT route.
constexpr int KMAX = 4096;
// Twiddle table tw[t] = exp(-2 pi i t / TWN), t = 0..TWN-1.
constexpr int TWN = 2 * KMAX;
// Largest GMRES basis handled by the device-side Givens kernel.
constexpr int MAX_ITER_CAP = 1000;
// Blocks used by the reduction kernels (partials per reduction).
constexpr int RED_BLOCKS = 608;  // 4 x 152 SMs

// Blocks of 256 threads for a vector kernel over n elements: about 8 elements a thread, at most
// RED_BLOCKS, so the kernels of a small problem leave the rest of the GPU to the problems running
// beside it (batched and served forms).  Producers and consumers of per-block partial sums use the
// same count.
__host__ __device__ inline int red_blocks(int64_t n) {
  const int64_t b = (n + 2047) / 2048;
  return b < 1 ? 1 : (b > RED_BLOCKS ? RED_BLOCKS : (int)b);
}

// FFT: n + 1 = K a power of two.  CHIRP: any n; the Toeplitz product uses a power-of-two circulant
// embedding of length 2K >= 2(n+1), the DST-I (two lines at a time) a Bluestein DFT of length n+1
// through a convolution of power-of-two length >= 2n.
// DENSE: explicit O(n) sums per output.  LONG (d = 1): lines longer than one CTA holds; the same
// convolutions as CHIRP, through four-step FFTs in global memory (tau_long.cu).
enum Route : int { ROUTE_FFT = 1, ROUTE_DENSE = 2, ROUTE_CHIRP = 3, ROUTE_LONG = 4 };


// What the value computed by a matvec pass becomes at the last dimension.
enum Finish : int {
  FIN_NONE = 0,    // out = value
  FIN_ADD_F = 1,   // out = value + Fdt            (right-hand side b)
  FIN_RESID = 2,   // out = src - value            (residual b - A x)
};

// What happens to the finished line before it is stored.
enum Post : int {
  POST_NONE = 0,
  POST_DST = 1,        // orthonormal DST-I along this dimension
  POST_DST_MU_DST = 2, // DST-I, multiply by 1/mu, DST-I  (only on dimension 0)
  POST_HT = 3,         // orthonormal Hartley transform along this dimension (dense, any n)
  POST_HT_D_HT = 4,    // Hartley, multiply by the diagonal in `invmu`, Hartley (only on dimension 0)
};

struct GmresDev;

// Double-float number: value = hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits, computed
// on the FP32 pipes.  Addition is Knuth's two-sum on the high parts followed by a renormalisation;
// multiplication uses the FMA-exact product of the high parts (Dekker, "A floating-point technique
// for extending the available precision", 1971; the FMA form of the product error).
struct __align__(8) df64 {
  float hi, lo;
};
struct __align__(16) df64x2 {
  df64 x, y;
};

template <typename T> struct Vec2Of;
template <> struct Vec2Of<double> { using type = double2; };
template <> struct Vec2Of<float> { using type = float2; };
template <> struct Vec2Of<df64> { using type = df64x2; };
template <typename T> using vec2 = typename Vec2Of<T>::type;

#ifdef __CUDACC__
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float h = s + e;
  return df64{h, e - (h - s)};
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64{-a.hi, -a.lo}; }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + df64{-b.hi, -b.lo}; }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float h = p + e;
  return df64{h, e - (h - p)};
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

// conversions (the double <-> float ones run on the FP64 pipe: keep them off inner loops)
template <typename T> __device__ __forceinline__ T from_d(double v) { return (T)v; }
template <> __device__ __forceinline__ df64 from_d<df64>(double v) {
  const float h = __double2float_rn(v);
  return df64{h, __double2float_rn(v - (double)h)};
}
template <typename T> __device__ __forceinline__ T from_f(float v) { return (T)v; }
template <> __device__ __forceinline__ df64 from_f<df64>(float v) { return df64{v, 0.0f}; }
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(df64 v) { return (double)v.hi + (double)v.lo; }
// element conversion between storage and compute types
template <typename T, typename S> __device__ __forceinline__ T cvt(S v) { return (T)v; }
template <> __device__ __forceinline__ df64 cvt<df64, double>(double v) { return from_d<df64>(v); }
template <> __device__ __forceinline__ df64 cvt<df64, df64>(df64 v) { return v; }
template <> __device__ __forceinline__ double cvt<double, df64>(df64 v) { return to_d(v); }
#endif

// Device tables of the long-line route for one dimension, in the element type T.  Both
// convolutions (Toeplitz product and chirp-z DST-I) have length F = 2 K_T (K_T the power of two
// >= n + 1), computed as F = F1 x F2 four-step FFTs over the array work[r * F2 + c] (natural
// index j = r F2 + c): F1-point DIFs down the columns, the twiddle tw4, F2-point DIFs along the
// rows; the spectrum ends at work[p1 * F2 + p2] = X[k1 + F1 k2] with p = dif_pos(k, .).
template <typename T>
struct LongTab {
  int n, F, F1, F2;
  int cw;                 // columns per CTA of the column kernels
  int lpr;                // rows per CTA of the row kernel
  const vec2<T>* tw1;     // stage-packed twiddles of the F1-point FFT (twp_size(F1))
  const vec2<T>* tw2;     // the same for F2
  const vec2<T>* tw4;     // [p1 * F2 + j2] = exp(-2 pi i j2 k1 / F), p1 = dif_pos(k1, F1)
  const vec2<T>* lam;     // Toeplitz circulant spectrum / F, in the spectrum layout
  const vec2<T>* bhat;    // chirp kernel spectrum * sqrt(2/L) / F (L = n + 1), same layout
  const vec2<T>* chirp;   // w_m = exp(i pi m^2 / (2L)), m = 0..n
  vec2<T>* work;          // F complex (scratch shared by the precisions of one problem)
  T* ybuf;                // n reals (scratch)
};

// Per-dimension data resident on the device, in the element type T of the pass (FP64 for the
// plain path, FP32 for the inner solve of the mixed-precision form).
template <typename T>
struct DimDataT {
  int n;              // interior points N_i
  int K;              // n + 1 (FFT route: power of two)
  int route;          // Route
  T bdiag, boff;      // B_{alpha_i}: 1 - alpha/12, alpha/24
  T dsc;              // sqrt(2 / K): scale of the orthonormal DST-I of length n
  double eta;         // kappa_i dt / (2 h_i^alpha_i)
  const vec2<T>* spec;  // FFT route: (a, b, c, d)_k, k = 0..K/2 (toep_pack_coeffs): the Toeplitz
                        // spectrum folded for the packed real FFT, scaled by 1/K (no eta)
  const T* s;           // FCD weights s_0..s_{n-1}
  const T* sintab;      // dense route: sin(pi t / K), t = 0..2K-1; FFT route: (1/2) sqrt(2/K) sin(pi t / K)
  const T* cas;         // Strang circulant method: cas(2 pi t / n) / sqrt(n), t = 0..n-1
  // CHIRP route DST-I: two lines share one DFT of length L = n+1 (the real-DFT form of the DST-I),
  // taken by Bluestein's method with c_m = exp(-i pi m^2 / L); M = convolution length (power of two
  // >= 2n: 2K, or K when n is a power of two)
  int M;
  const vec2<T>* chirp;  // c_m, m = 0..n
  const vec2<T>* bhat;   // FFT_M of conj(c_|m|) placed at m mod M, in the digit-reversed order fft_dif
                         // leaves, times sqrt(2/L)/(2M)
  const vec2<T>* twM;    // stage-packed twiddles of the length-M FFT
  const vec2<T>* twK;   // FFT route: stage-packed twiddles of the length-K FFT, then W (see twp_size)
  const vec2<T>* twK2;  // FFT route: the same for the length-K/2 FFT of the DST-I
  const LongTab<T>* lng;  // LONG route: host pointer to the dimension's tables (not read on the device)
};
using DimData = DimDataT<double>;

// Stage-packed twiddle table of an in-place radix-4 FFT of length S (twp_size(S) entries):
//   stage of size s (s = S, S/4, ..., >= 4) at offset S - s: [w_s^i | w_s^{2i} | w_s^{3i}], i < s/4,
//   with w_s = exp(-2 pi i / s); then at offset S: exp(-2 pi i k / (2S)), k = 0..S.
// Consecutive butterflies of a stage read consecutive entries.
__host__ __device__ inline int twp_size(int S) { return 2 * S + 1; }

// Coefficients (a, b, c, d) of the spectral step of the Toeplitz product for the pair (k, K-k):
// with Z the packed half-length DFT of the zero-padded line, Z'_k = a Z_k + b conj(Z_{K-k}) and
// Z'_{K-k} = c conj(Z_k) + d Z_{K-k}.  The map unpacks the length-2K real DFT at k,
// Y_k = (E + W_k O)/2 with E = Z_k + conj Z_{K-k}, O = -i (Z_k - conj Z_{K-k}) and
// W_k = (wx, wy) = exp(-i pi k / K), multiplies by lambda_k, lambda_{K-k} and repacks for the
// unnormalised inverse (1/K); it is evaluated on the basis inputs (Z_k, Z_{K-k}) = (1, 0), (0, 1).
// out: 8 reals (a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y).
__host__ __device__ inline void toep_pack_coeffs(double lk, double lkk, double wx, double wy, int K, double* out) {
  const double sg = (lk + lkk) / (4.0 * K), dl = (lk - lkk) / (4.0 * K);
  for (int basis = 0; basis < 2; ++basis) {
    const double ax = basis == 0 ? 1.0 : 0.0, bx = basis == 1 ? 1.0 : 0.0;   // imaginary parts 0
    const double e2x = ax + bx, e2y = 0.0;
    const double o2x = 0.0, o2y = bx - ax;
    const double px = wx * o2x - wy * o2y, py = wx * o2y + wy * o2x;
    const double epx = sg * e2x + dl * px, epy = sg * e2y + dl * py;
    const double wcx = e2x * wx + e2y * wy, wcy = e2y * wx - e2x * wy;
    const double opx = dl * wcx + sg * o2x, opy = dl * wcy + sg * o2y;
    // basis 0 gives a (Z'_k) and c (Z'_{K-k}); basis 1 gives b and d
    out[2 * basis + 0] = epx - opy;
    out[2 * basis + 1] = epy + opx;
    out[4 + 2 * basis + 0] = epx + opy;
    out[4 + 2 * basis + 1] = opx - epy;
  }
}

// One line pass over an array of shape (n_{d-1}, ..., n_0) along dimension ax.
template <typename T>
struct PassT {
  int ax;            // dimension (0 = x_1, contiguous)
  int len;           // n_ax
  int64_t inner;     // prod_{i<ax} n_i (element stride along the line)
  int64_t nlines;    // n_tot / len
  int lpb;           // lines per CTA
  int tpb;           // threads per CTA: 128 (0 means 128) or 256 (the wide variant)
  int64_t ntiles;
  DimDataT<T> dim;
  // matvec channels
  int mv;            // 1: this pass is a matvec pass
  int first;         // 1: inputs are (x, e): a = B(e∘x) + s eta T x, c = B x
  int last;          // 1: no c output; apply Finish
  double seta;       // +eta (A) or -eta (right-hand side)
  int toep_only;     // 1: out = T x (no B, no eta) -- Toeplitz parity entry
  int finish;        // Finish
  int post;          // Post
  const T* in_a;        // first pass: x; else channel a
  const T* in_c;        // channel c (not read by the first pass)
  const T* e;           // first pass: e at the interior nodes
  const T* src;         // FIN_RESID minuend or FIN_ADD_F addend (Fdt)
  const T* invmu;       // POST_DST_MU_DST
  T* out_a;
  T* out_c;
  // Krylov wiring: pointers that depend on the device-side Arnoldi index j
  const GmresDev* g;    // non-null: skip the pass when g->done
  const int* skip;      // non-null: skip the pass when *skip != 0
  T* in_base;           // in_sel: 1 -> in_base + j*vstride, 2 -> in_base + (j+1)*vstride
  T* out_base;          // out_sel: the same for the output
  int64_t vstride;
  int in_sel, out_sel;  // 0: in_a/out_a as given
};
using Pass = PassT<double>;

// GMRES state kept in device memory (one per problem).
struct GmresDev {
  int j;             // current Arnoldi index: V_j is the newest basis vector
  int done;          // 1 once converged / capped / broken down
  int k;             // iterations of the finished step
  int notconv;       // sticky: some step hit max_iter
  int max_iter;
  unsigned int tickets;  // last-block counter of the fused Gram-Schmidt reductions (0 between launches)
  double tol;
  double beta;       // ||r_0||
  double relres;
  double hnorm;      // ||w|| of the current column
  int64_t m;         // current step index
  int64_t M;
};

// ---------------------------------------------------------------------------
// host launchers (tau_kernels.cu)
// ---------------------------------------------------------------------------
cudaError_t init_kernel_attributes();
// Message returned by tau_last_error() for the calling thread.
void set_last_error(const char* msg);
template <typename T> size_t pass_smem_bytes(const PassT<T>& p);
template <typename T> cudaError_t launch_pass(const PassT<T>& p, cudaStream_t st);
cudaError_t launch_spectrum(int K, const double* c, double* lam, const double2* twK, cudaStream_t st);
// out[p] = scale * (DFT_M b) in the digit-reversed layout of fft_dif (one block, M <= 8192)
cudaError_t launch_chirp_spectrum(int M, const double2* b, double2* out, const double2* twM, double scale,
                                  cudaStream_t st);
// Fill a stage-packed twiddle table (twp_size(S) entries) on the device.
cudaError_t launch_twp(int S, double2* twp, cudaStream_t st);

// tensor-core DST-I mode product of the FP32 τ solve (tau_tc.cu), one dimension with n <= 256
struct TcTab {
  int n;          // line length
  int N;          // rows of T: n rounded up to 128 on dimension 0, to 16 elsewhere
  int Kp16;       // n rounded up to 16 (shared-memory K chunks of both kernels)
  int nalloc;     // TMEM columns of the matvec (power of two >= max(32, N))
  int Nh;         // rows of the half DST matrix: 128 on dimension 0, else ceil(n/2) rounded up to 16
  int nalloc_h;   // TMEM columns of the DST (two accumulators: even and odd j)
  const float* S; // rows 0..ceil(n/2)-1 of the orthonormal DST-I matrix, TF32-rounded, zero padded to
                  // Nh x Kp16, per K-chunk of 16 columns in the core-matrix layout (512-byte row
                  // groups), the chunk's even columns in slots 0-7 and its odd ones in slots 8-15
  CUtensorMap tmS; // S as a 2-D tensor of 256-value rows, a box (Nh / 16 rows) per K-chunk: the tiled
                   // bulk copy (TMA) of a chunk
  int* err;       // device flag: an mbarrier wait gave up
  // split-TF32 Toeplitz matvec: T_ax (FCD weights) = T_hi + T_lo, zero padded to N x Kp16, stored
  // per K-chunk of 16 columns in the same layout; tmThi, tmTlo: their tensor maps (box = one chunk)
  const float* Thi;
  const float* Tlo;
  CUtensorMap tmThi, tmTlo;
};
cudaError_t init_tc_attributes();
// one CTA waits (bounded, `polls` polls) on an mbarrier nothing arrives at; *gave_up = 1 when the
// wait gave up as it must
cudaError_t launch_wait_selftest(int polls, int* gave_up, cudaStream_t st);
// y = S x along p.ax for every line (from_out: x is p's output, in place); mul: optional diagonal
// applied to the result
cudaError_t launch_tc_dst(const PassT<float>& p, const TcTab& t, const float* mul, bool from_out, cudaStream_t st);
// One matvec pass along p.ax with T c on the tensor cores (split TF32): a' = B a + seta T c,
// c' = B c (not last); first: a = e∘x, c = x (c_in, optionally device-selected); last: a' to out
cudaError_t launch_tc_mv(const PassT<float>& p, const TcTab& t, const float* c_in, float* c_base, int c_sel,
                         const float* a_in, float* out_a, float* out_base, int out_sel, float* out_c, bool first,
                         bool last, cudaStream_t st);

// next right-hand side of the mixed form from the last residual (tau_mixed.cu); every kernel returns
// at once when *flag == 0.  save: y = E∘u; rhs: y += E'∘u, b = B y + r - b + fdt (B the d-level
// tridiagonal product with bd, bo per dimension, applied one factor at a time through y2, which it
// overwrites along with y); set_flag: *flag = v.
cudaError_t launch_rres_save(const int* flag, const double* E, const double* u, double* y, int64_t n,
                             cudaStream_t st);
cudaError_t launch_rres_rhs(const int* flag, int d, const int* nn, const double* bd, const double* bo,
                            const double* E, const double* u, double* y, double* y2, const double* r, int r_df,
                            double* b, const double* fdt, int64_t n, cudaStream_t st);
cudaError_t launch_set_flag(int* flag, int v, cudaStream_t st);

// long-line route (tau_long.cu)
cudaError_t init_long_attributes();
// One line pass (the semantics of launch_pass for d = 1) as a sequence of four-step FFT launches.
template <typename T> cudaError_t launch_long(const PassT<T>& p, const LongTab<T>& L, cudaStream_t st);
// Kernels launch_long enqueues for the pass p.
template <typename T> int long_launches(const PassT<T>& p);
// Setup: tw4 of (F1, F2); the forward four-step FFT of src (F complex, natural order) scaled by
// `scale` into dst (spectrum layout; work is overwritten); q_k = s_0 + 2 sum_j s_j cos(pi j k/(n+1))
// with ct[t] = cos(pi t / (n+1)), t < 2(n+1).
cudaError_t launch_long_tw4(int F1, int F2, double2* tw4, cudaStream_t st);
cudaError_t launch_long_spectrum(const LongTab<double>& L, const double2* src, double2* dst, double scale,
                                 cudaStream_t st);
cudaError_t launch_q_direct(int n, const double* s, const double* ct, double* q, cudaStream_t st);

// fields: e_m, Fdt_m for step m (read from g->m unless m_override >= 0)
struct FieldDev {
  int d;
  int n[3];
  int64_t n_tot;
  int re, rf;                 // ranks of e and f
  const double* e_tc;         // [M x re]
  const double* e_sp[3];      // [re x (n_i+2)]
  const double* f_tc;         // [M x rf]
  const double* f_hsp[3];     // [rf x n_i]: 𝓗-stencilled f space tables (interior)
  double dt;
  // dense form (tau_set_fields_device; the tables above are unused when e_dev is set): e at the
  // interior nodes, step m at e_dev + m * e_step; f on the padded grid prod (n_i + 2), step m at
  // f_dev + m * f_step (NULL: f = 0); a step of 0 means the field does not depend on t
  const double* e_dev;
  int64_t e_step;
  const double* f_dev;
  int64_t f_step;
  double hw[3][2];            // 𝓗_{alpha_i} stencil weights: (alpha_i/24, 1 - alpha_i/12)
};
cudaError_t launch_fields(const FieldDev& f, const GmresDev* g, int64_t m_override, double* e_out,
                          double* fdt_out, cudaStream_t st);
cudaError_t launch_psi(int d, const int* n, int64_t n_tot, int rank, const double* tc, const double* const* sp,
                       double* out, cudaStream_t st);
cudaError_t launch_escan(const FieldDev& f, int64_t M, double* partial /*2*RED_BLOCKS*/, cudaStream_t st);
cudaError_t launch_invmu(int d, const int* n, int64_t n_tot, double ebar, const double* const* beta,
                         const double* const* q, const double* eta, double* invmu, cudaStream_t st);
// Two-sided preconditioning (Eq. (Pls)): pmh = sqrt(beta/mu), pmhb = 1/sqrt(beta mu) per sine mode.
cudaError_t launch_tpgm_diag(int d, const int* n, int64_t n_tot, double ebar, const double* const* beta,
                             const double* const* q, const double* eta, double* pmh, double* pmhb, cudaStream_t st);
// Strang circulant method (Eq. (Pcir)): pcinv = 1/p_k with p_k = ebar + c(S)_k / c(B)_k on the
// Fourier basis (bs, ss: per-dimension DFT eigenvalues of s(B_i), s(S_i)); binv = 1/prod_i beta_k
// (B^{-1} on the sine basis).
cudaError_t launch_spgm_diag(int d, const int* n, int64_t n_tot, double ebar, const double* const* bs,
                             const double* const* ss, const double* eta, const double* const* beta, double* pcinv,
                             double* binv, cudaStream_t st);
// u = t (keep 0) or u += t (keep 1)
cudaError_t launch_add_into(double* u, const double* t, int64_t n, int keep, cudaStream_t st);

// GMRES building blocks
// w = V_{j+1} (the slot of the next basis vector) in the CGS2 kernels below; S is the storage
// type of the basis (products in S, reductions in FP64).  Each kernel's per-block partial sums are
// finished by the block that completes last (a ticket counter in GmresDev), so a CGS2 iteration is
// three launches: h1 = V^T w; w -= V h1 and h2 = V^T w; w -= V h2, ||w|| and the Givens column.
template <typename S>
cudaError_t launch_dots(const S* V, int64_t n, GmresDev* g, double* partial, int ld_partial, double* h,
                        cudaStream_t st);
template <typename S>
cudaError_t launch_update_dots(S* V, int64_t n, GmresDev* g, const double* h_in, double* partial, int ld_partial,
                               double* h_out, cudaStream_t st);
// Arguments of the Givens step that closes an Arnoldi column (Hessenberg column j = h1 + h2 and
// ||w||, rotations, residual estimate, stop test, graph condition).
struct GivensArgs {
  double* H;
  double* cs;
  double* sn;
  double* gv;
  const double* h1;
  const double* h2;
  int ldH;
  int use_cond;        // 0 none, 1 this problem's handle, 2 a group's (gc)
  cudaGraphConditionalHandle cond;
  GroupCtl* gc;
};
template <typename S>
cudaError_t launch_update_norm_givens(S* V, int64_t n, GmresDev* g, const double* h2, double* partial_norm,
                                      const GivensArgs& ga, cudaStream_t st);
template <typename S>
cudaError_t launch_scale_next(S* V, int64_t n, const GmresDev* g, cudaStream_t st);
template <typename S>
cudaError_t launch_norm_partial(const S* w, int64_t n, const GmresDev* g, double* partial, cudaStream_t st);
template <typename S>
cudaError_t launch_init_beta(GmresDev* g, const double* partial, double* gv, S* V, int64_t n, cudaStream_t st);
template <typename S>
cudaError_t launch_backsolve_update(GmresDev* g, const double* H, const double* gv, int ldH, double* y, const S* V,
                                    int64_t n, S* u, int x0_prev, int* iters_log, cudaStream_t st);
cudaError_t launch_d_to_df(const double* a, df64* b, int64_t n, cudaStream_t st);
cudaError_t launch_df_to_d(const df64* a, double* b, int64_t n, cudaStream_t st);
cudaError_t launch_fp64_peak(double* out, int blocks, int iters, cudaStream_t st);

// Iterative-refinement state of the mixed-precision form (device memory).
struct IRDev {
  int sweep;         // corrections applied so far in this step
  int done;
  int max_sweeps;
  int notconv;       // sticky: some step stopped at max_sweeps
  int inner_total;   // inner FGMRES iterations of this step
  int skip_resid;    // 1 while the first residual of a step equals b (zero initial guess)
  double tol;        // ||b - A x|| <= tol ||b - A x_0||
  double rho0, rho, last_rel;
  double inner_tol;  // inner FGMRES target of the first sweep (later sweeps: k_ir_control)
  double rho_prev;   // residual norm before the last correction
  double itol_prev;  // inner target of the last sweep
};
cudaError_t launch_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t st);
cudaError_t launch_ir_init(IRDev* ir, cudaStream_t st);
// Residual of the zero initial guess: r = b on the first sweep (the FP64 residual passes are
// skipped through ir->skip_resid); later sweeps compute b - A x.
cudaError_t launch_ir_first_resid(IRDev* ir, const double* b, double* r, int64_t n, int x0_zero, cudaStream_t st);
cudaError_t launch_ir_control(IRDev* ir, GmresDev* gin, double* gv_in, const double* pnorm, int64_t n,
                              cudaGraphConditionalHandle cond, cudaGraphConditionalHandle cond_in, int use_cond,
                              GroupCtl* gc, cudaStream_t st);
// dst = src (src non-null) or dst = 0, n doubles (a kernel, so it can be recorded and grouped)
cudaError_t launch_copy(double* dst, const double* src, int64_t n, cudaStream_t st);
// v = r / rho in FP32 from the residual stored as S (double, or double-float)
template <typename S>
cudaError_t launch_scale_to_f32(const S* r, float* v, int64_t n, const IRDev* ir, cudaStream_t st);
// x += rho sum_i y_i Z_i (the sum in FP64) with x stored as X (double, or double-float)
template <typename X>
cudaError_t launch_update_x(X* x, const float* Z, const double* y, int64_t n, const GmresDev* gin, IRDev* ir,
                            cudaStream_t st);
cudaError_t launch_ir_finish(const IRDev* ir, GmresDev* g, int* iters_log, int* sweeps_log, cudaStream_t st);
cudaError_t launch_backsolve(GmresDev* g, const double* H, const double* gv, int ldH, double* y, cudaStream_t st);

}  // namespace tau
