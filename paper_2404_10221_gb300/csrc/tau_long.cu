// Long-line route (d = 1, lines longer than one CTA's shared memory holds).
//
// A line pass of the one-dimensional problem -- the matvec y = B(e∘x) + s eta T x of Eq. (tls)
// with its finish, the Toeplitz product alone, the orthonormal DST-I and the DST-I·diag·DST-I of
// the τ solve (Eqs. (Pa), (diag)) -- is the same arithmetic as on the chirp route, but its two
// convolutions run as four-step FFTs over an array in global memory (L2-resident at these sizes)
// instead of in one CTA:
//
//   Toeplitz product  T x = first n entries of IFFT_F(lambda ∘ FFT_F(x zero-padded)), F = 2 K_T,
//                     lambda the spectrum of the circulant embedding of the FCD weights s_k;
//   DST-I             y_k = sqrt(2/L) Im(w_k z_{k-1}), z = circular convolution (length F >= 2n) of
//                     a_m = w_{m+1} x_{m+1} with conj(w_|m|), w_m = exp(i pi m^2 / (2L)), L = n + 1
//                     (jk = (j^2 + k^2 - (k-j)^2)/2 turns the sine sum into a convolution).
//
// Four-step FFT of length F = F1 F2 on work[r F2 + c] (natural index j = r F2 + c): F1-point
// decimation-in-frequency FFTs down the F2 columns, a multiply by exp(-2 pi i c k1 / F), F2-point
// DIFs along the F1 rows.  The spectrum is left in the digit-reversed layout both DIFs produce; the
// pointwise products use spectra stored in that layout, and the inverse runs the mirrored
// decimation-in-time steps (rows, conjugate twiddle, columns), so no transposition is needed.
// One convolution is three launches: column DIF (its input stage fused: zero padding or the chirp
// multiply), row DIF + pointwise product + row DIT, column DIT (its output stage fused: the real
// part with the matvec stencil and finish, or the chirp demodulation and the diagonal).
#include "tau_internal.cuh"
#include "tau_fft.cuh"

#include <math.h>

#include <type_traits>

namespace tau {

constexpr int LONG_THREADS = 128;

enum ColIn : int { CIN_RAW = 0, CIN_TOEP = 1, CIN_CHIRP = 2 };
enum ColOut : int { COUT_TOEP = 1, COUT_CHIRP = 2 };
enum RowMode : int { ROW_FWD = 0, ROW_CONV = 1 };

template <typename T>
struct LongArgs {
  int n, F1, F2, lgF2, cw, lgcw, lpr;
  const vec2<T>* tw1;
  const vec2<T>* tw2;
  const vec2<T>* tw4;
  const vec2<T>* chirp;
  const vec2<T>* spec;   // row kernel: lam or bhat
  vec2<T>* work;
  const T* in;           // forward column kernel input (and x of the matvec stencil)
  T* in_base;
  int in_sel;
  T* out;                // inverse column kernel output
  T* out_base;
  int out_sel;
  int64_t vstride;
  const GmresDev* g;
  const int* skip;
  int mv;                // inverse Toeplitz output: B(e∘x) + seta * (T x), then finish
  const T* e;
  T bd, bo;
  double seta;
  int finish;
  const T* src;
  const T* mul;          // inverse chirp output: multiply by this diagonal (null: none)
};

template <typename T>
__device__ __forceinline__ bool long_skip(const LongArgs<T>& a) {
  return (a.g && a.g->done) || (a.skip && *a.skip);
}
template <typename T>
__device__ __forceinline__ const T* long_in(const LongArgs<T>& a) {
  return a.in_sel ? a.in_base + (int64_t)(a.g->j + a.in_sel - 1) * a.vstride : a.in;
}
template <typename T>
__device__ __forceinline__ T* long_out(const LongArgs<T>& a) {
  return a.out_sel ? a.out_base + (int64_t)(a.g->j + a.out_sel - 1) * a.vstride : a.out;
}

// Column DIF: CTA b owns columns c0 = b*cw .. c0+cw-1, held as cw lines of F1 complex in shared
// memory; the twiddle is applied on the way out.  CIN_TOEP / CIN_CHIRP inputs are zero at natural
// indices >= n <= F/2, i.e. in rows >= F1/2, which the first DIF stage then skips.
template <typename T, int IN>
__global__ void __launch_bounds__(LONG_THREADS) k_long_col_fwd(const LongArgs<T> a) {
  using V = vec2<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* cb = reinterpret_cast<V*>(smraw);
  if (long_skip(a)) return;
  const int F1 = a.F1, F2 = a.F2, cw = a.cw, lgcw = a.lgcw;
  const int c0 = blockIdx.x * cw;
  const int tid = threadIdx.x, TH = blockDim.x;
  const bool zero_hi = IN != CIN_RAW && F1 >= 4;
  const int rows = zero_hi ? F1 >> 1 : F1;
  const T* x = IN == CIN_RAW ? nullptr : long_in(a);
  const V z0 = mk<V>(from_f<T>(0.0f), from_f<T>(0.0f));
  for (int idx = tid; idx < (rows << lgcw); idx += TH) {
    const int r = idx >> lgcw, l = idx & (cw - 1);
    const int64_t j = (int64_t)r * F2 + c0 + l;
    V v;
    if constexpr (IN == CIN_RAW) {
      v = a.work[j];
    } else if constexpr (IN == CIN_TOEP) {
      v = j < a.n ? mk<V>(x[j], from_f<T>(0.0f)) : z0;
    } else {
      v = z0;
      if (j < a.n) {
        const V w = ldt(&a.chirp[j + 1]);
        const T xv = x[j];
        v = mk<V>(xv * w.x, xv * w.y);
      }
    }
    cb[l * F1 + r] = v;
  }
  __syncthreads();
  fft_dif(cb, F1, cw, F1, a.tw1, zero_hi);
  for (int idx = tid; idx < (F1 << lgcw); idx += TH) {
    const int p = idx >> lgcw, l = idx & (cw - 1);
    const int64_t o = (int64_t)p * F2 + c0 + l;
    a.work[o] = cmul(cb[l * F1 + p], ldt(&a.tw4[o]));
  }
}

// Rows: CTA b owns rows r0 = b*lpr .. r0+lpr-1.  ROW_FWD: DIF only (setup); ROW_CONV: DIF, product
// with the spectrum, unnormalised inverse DIT (the spectrum carries 1/F).
template <typename T, int MODE>
__global__ void __launch_bounds__(LONG_THREADS) k_long_row(const LongArgs<T> a) {
  using V = vec2<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* cb = reinterpret_cast<V*>(smraw);
  if (long_skip(a)) return;
  const int F2 = a.F2, lpr = a.lpr;
  const int64_t base = (int64_t)blockIdx.x * lpr * F2;
  const int tid = threadIdx.x, TH = blockDim.x;
  const int tot = lpr * F2;
  for (int idx = tid; idx < tot; idx += TH) cb[idx] = a.work[base + idx];
  __syncthreads();
  fft_dif(cb, F2, lpr, F2, a.tw2);
  if constexpr (MODE == ROW_CONV) {
    for (int idx = tid; idx < tot; idx += TH) cb[idx] = cmul(cb[idx], ldt(&a.spec[base + idx]));
    __syncthreads();
    fft_dit<true>(cb, F2, lpr, F2, a.tw2);
  }
  for (int idx = tid; idx < tot; idx += TH) a.work[base + idx] = cb[idx];
}

// Column DIT (inverse): conjugate twiddle on the way in, F1-point inverse DIT down the columns, then
// the output stage for natural indices j < n (rows < F1/2: half_out).
template <typename T, int OUT>
__global__ void __launch_bounds__(LONG_THREADS) k_long_col_inv(const LongArgs<T> a) {
  using V = vec2<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* cb = reinterpret_cast<V*>(smraw);
  if (long_skip(a)) return;
  const int F1 = a.F1, F2 = a.F2, cw = a.cw, lgcw = a.lgcw, n = a.n;
  const int c0 = blockIdx.x * cw;
  const int tid = threadIdx.x, TH = blockDim.x;
  for (int idx = tid; idx < (F1 << lgcw); idx += TH) {
    const int p = idx >> lgcw, l = idx & (cw - 1);
    const int64_t o = (int64_t)p * F2 + c0 + l;
    cb[l * F1 + p] = cmulc(a.work[o], ldt(&a.tw4[o]));
  }
  __syncthreads();
  const bool half = F1 >= 4;
  fft_dit<true>(cb, F1, cw, F1, a.tw1, half);
  const int rows = half ? F1 >> 1 : F1;
  T* out = long_out(a);
  const T* x = (OUT == COUT_TOEP && a.mv) ? long_in(a) : nullptr;
  const T zero = from_f<T>(0.0f);
  for (int idx = tid; idx < (rows << lgcw); idx += TH) {
    const int r = idx >> lgcw, l = idx & (cw - 1);
    const int64_t j = (int64_t)r * F2 + c0 + l;
    if (j >= n) continue;
    const V z = cb[l * F1 + r];
    T val;
    if constexpr (OUT == COUT_TOEP) {
      val = z.x;
      if (a.mv) {
        // B(e∘x) at j (Eq. (tls)), neighbours read from global memory
        const T ex = a.e[j] * x[j];
        const T lft = j > 0 ? a.e[j - 1] * x[j - 1] : zero;
        const T rgt = j + 1 < n ? a.e[j + 1] * x[j + 1] : zero;
        const T ba = tfma(a.bd, ex, a.bo * (lft + rgt));
        val = tfma(from_d<T>(a.seta), val, ba);
        if (a.finish == FIN_ADD_F) val = val + a.src[j];
        else if (a.finish == FIN_RESID) val = a.src[j] - val;
      }
    } else {
      const V w = ldt(&a.chirp[j + 1]);
      val = tfma(w.x, z.y, w.y * z.x);   // Im(w_{j+1} z_j)
      if (a.mul) val = val * a.mul[j];
    }
    out[j] = val;
  }
}

template <typename T>
__global__ void k_long_copy(const LongArgs<T> a) {
  if (long_skip(a)) return;
  const T* x = long_in(a);
  T* y = long_out(a);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x)
    y[j] = x[j];
}

template <typename T>
size_t col_smem(const LongArgs<T>& a) {
  return (size_t)a.cw * a.F1 * sizeof(vec2<T>);
}
template <typename T>
size_t row_smem(const LongArgs<T>& a) {
  return (size_t)a.lpr * a.F2 * sizeof(vec2<T>);
}

template <typename T, int IN>
cudaError_t col_fwd(const LongArgs<T>& a, cudaStream_t st) {
  k_long_col_fwd<T, IN><<<a.F2 / a.cw, LONG_THREADS, col_smem(a), st>>>(a);
  return cudaGetLastError();
}
template <typename T, int MODE>
cudaError_t row_pass(const LongArgs<T>& a, cudaStream_t st) {
  k_long_row<T, MODE><<<a.F1 / a.lpr, LONG_THREADS, row_smem(a), st>>>(a);
  return cudaGetLastError();
}
template <typename T, int OUT>
cudaError_t col_inv(const LongArgs<T>& a, cudaStream_t st) {
  k_long_col_inv<T, OUT><<<a.F2 / a.cw, LONG_THREADS, col_smem(a), st>>>(a);
  return cudaGetLastError();
}

template <typename T>
LongArgs<T> long_args(const PassT<T>& p, const LongTab<T>& L) {
  LongArgs<T> a{};
  a.n = L.n;
  a.F1 = L.F1;
  a.F2 = L.F2;
  a.lgF2 = 0;
  while ((1 << a.lgF2) < L.F2) ++a.lgF2;
  a.cw = L.cw;
  a.lgcw = 0;
  while ((1 << a.lgcw) < L.cw) ++a.lgcw;
  a.lpr = L.lpr;
  a.tw1 = L.tw1;
  a.tw2 = L.tw2;
  a.tw4 = L.tw4;
  a.chirp = L.chirp;
  a.work = L.work;
  a.vstride = p.vstride;
  a.g = p.g;
  a.skip = p.skip;
  a.bd = p.dim.bdiag;
  a.bo = p.dim.boff;
  a.seta = p.seta;
  a.e = p.e;
  a.src = p.src;
  a.finish = p.finish;
  return a;
}

#define LTRY(x)                                   \
  do {                                            \
    const cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) return e_;             \
  } while (0)

// One chirp-z DST-I of a.in (resolved) into a.out (resolved), times a.mul if set.
template <typename T>
cudaError_t long_dst(LongArgs<T> a, const LongTab<T>& L, cudaStream_t st) {
  a.spec = L.bhat;
  LTRY((col_fwd<T, CIN_CHIRP>(a, st)));
  LTRY((row_pass<T, ROW_CONV>(a, st)));
  return col_inv<T, COUT_CHIRP>(a, st);
}

template <typename T>
cudaError_t launch_long(const PassT<T>& p, const LongTab<T>& L, cudaStream_t st) {
  const LongArgs<T> base = long_args(p, L);
  // stage 1 input: the pass input as given (device-selected vectors resolved in the kernels)
  LongArgs<T> in = base;
  in.in = p.in_a;
  in.in_base = p.in_base;
  in.in_sel = p.in_sel;
  // final output
  auto to_out = [&](LongArgs<T>& a) {
    a.out = p.out_a;
    a.out_base = p.out_base;
    a.out_sel = p.out_sel;
  };
  auto to_ybuf = [&](LongArgs<T>& a) {
    a.out = L.ybuf;
    a.out_base = nullptr;
    a.out_sel = 0;
  };
  auto from_ybuf = [&](LongArgs<T>& a) {
    a.in = L.ybuf;
    a.in_base = nullptr;
    a.in_sel = 0;
  };
  const bool dst = p.post == POST_DST || p.post == POST_DST_MU_DST;
  if (p.post != POST_NONE && !dst) return cudaErrorNotSupported;   // Hartley passes: not on this route
  if (p.mv || p.toep_only) {
    // matvec (or Toeplitz product): the stencil reads x at j-1, j, j+1 while outputs are written,
    // so an output that aliases the input goes through ybuf
    const bool alias = !p.in_sel && !p.out_sel && p.in_a == p.out_a;
    LongArgs<T> a = in;
    a.mv = p.mv;
    a.spec = L.lam;
    LTRY((col_fwd<T, CIN_TOEP>(a, st)));
    LTRY((row_pass<T, ROW_CONV>(a, st)));
    if (dst || alias) to_ybuf(a);
    else to_out(a);
    LTRY((col_inv<T, COUT_TOEP>(a, st)));
    if (!dst) {
      if (!alias) return cudaSuccess;
      LongArgs<T> c = base;
      from_ybuf(c);
      to_out(c);
      k_long_copy<T><<<red_blocks(L.n), 256, 0, st>>>(c);
      return cudaGetLastError();
    }
    from_ybuf(in);
  } else if (!dst) {
    LongArgs<T> c = in;
    to_out(c);
    k_long_copy<T><<<red_blocks(L.n), 256, 0, st>>>(c);
    return cudaGetLastError();
  }
  // in: the DST input (the pass input, or ybuf after a matvec)
  if (p.post == POST_DST) {
    LongArgs<T> a = in;
    to_out(a);
    return long_dst(a, L, st);
  }
  // DST, times the diagonal, DST: the first result goes to ybuf (the forward column kernel has
  // consumed its input before the inverse column kernel writes)
  LongArgs<T> a = in;
  to_ybuf(a);
  a.mul = p.invmu;
  LTRY(long_dst(a, L, st));
  LongArgs<T> b = base;
  from_ybuf(b);
  to_out(b);
  return long_dst(b, L, st);
}

template <typename T>
int long_launches(const PassT<T>& p) {
  const bool dst = p.post == POST_DST || p.post == POST_DST_MU_DST;
  int k = 0;
  if (p.mv || p.toep_only) {
    k = 3;
    if (!dst && !p.in_sel && !p.out_sel && p.in_a == p.out_a) k += 1;   // copy out of ybuf
  } else if (!dst) {
    k = 1;
  }
  if (p.post == POST_DST) k += 3;
  if (p.post == POST_DST_MU_DST) k += 6;
  return k;
}

template int long_launches<double>(const PassT<double>&);
template int long_launches<float>(const PassT<float>&);
template int long_launches<df64>(const PassT<df64>&);
template cudaError_t launch_long<double>(const PassT<double>&, const LongTab<double>&, cudaStream_t);
template cudaError_t launch_long<float>(const PassT<float>&, const LongTab<float>&, cudaStream_t);
template cudaError_t launch_long<df64>(const PassT<df64>&, const LongTab<df64>&, cudaStream_t);

cudaError_t init_long_attributes() {
  const int lim = 200 * 1024;
#define LATTR(k) LTRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))
  LATTR((k_long_col_fwd<double, CIN_RAW>));
  LATTR((k_long_col_fwd<double, CIN_TOEP>));
  LATTR((k_long_col_fwd<double, CIN_CHIRP>));
  LATTR((k_long_col_fwd<float, CIN_TOEP>));
  LATTR((k_long_col_fwd<float, CIN_CHIRP>));
  LATTR((k_long_col_fwd<df64, CIN_TOEP>));
  LATTR((k_long_col_fwd<df64, CIN_CHIRP>));
  LATTR((k_long_row<double, ROW_FWD>));
  LATTR((k_long_row<double, ROW_CONV>));
  LATTR((k_long_row<float, ROW_CONV>));
  LATTR((k_long_row<df64, ROW_CONV>));
  LATTR((k_long_col_inv<double, COUT_TOEP>));
  LATTR((k_long_col_inv<double, COUT_CHIRP>));
  LATTR((k_long_col_inv<float, COUT_TOEP>));
  LATTR((k_long_col_inv<float, COUT_CHIRP>));
  LATTR((k_long_col_inv<df64, COUT_TOEP>));
  LATTR((k_long_col_inv<df64, COUT_CHIRP>));
#undef LATTR
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
__global__ void k_long_tw4(int F1, int F2, double2* tw4) {
  const int64_t F = (int64_t)F1 * F2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < F; t += (int64_t)gridDim.x * blockDim.x) {
    const int k1 = (int)(t / F2), j2 = (int)(t - (int64_t)k1 * F2);
    const int64_t r = ((int64_t)j2 * k1) % F;   // exact phase index
    double sv, cv;
    sincospi(-2.0 * (double)r / (double)F, &sv, &cv);
    tw4[(int64_t)dif_pos(k1, F1) * F2 + j2] = make_double2(cv, sv);
  }
}

cudaError_t launch_long_tw4(int F1, int F2, double2* tw4, cudaStream_t st) {
  const int64_t F = (int64_t)F1 * F2;
  k_long_tw4<<<(unsigned)((F + 255) / 256 < 4096 ? (F + 255) / 256 : 4096), 256, 0, st>>>(F1, F2, tw4);
  return cudaGetLastError();
}

__global__ void k_long_scale(const double2* __restrict__ a, double2* b, int64_t F, double scale) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < F; t += (int64_t)gridDim.x * blockDim.x)
    b[t] = make_double2(scale * a[t].x, scale * a[t].y);
}

cudaError_t launch_long_spectrum(const LongTab<double>& L, const double2* src, double2* dst, double scale,
                                 cudaStream_t st) {
  const int64_t F = (int64_t)L.F;
  LTRY(cudaMemcpyAsync(L.work, src, (size_t)F * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  PassT<double> p{};
  LongArgs<double> a = long_args(p, L);
  LTRY((col_fwd<double, CIN_RAW>(a, st)));
  LTRY((row_pass<double, ROW_FWD>(a, st)));
  const unsigned blocks = (unsigned)((F + 255) / 256 < 4096 ? (F + 255) / 256 : 4096);
  k_long_scale<<<blocks, 256, 0, st>>>(L.work, dst, F, scale);
  return cudaGetLastError();
}

// q_k = s_0 + 2 sum_{j=1}^{n-1} s_j cos(pi j k / L), k = 1..n (Eq. (q)), one thread per k; the
// angle index j k is reduced modulo 2L exactly and looked up in ct[t] = cos(pi t / L), t < 2L.
// Summed in the order the equation is written (s_0, then j ascending), each term 2 s_j cos rounded
// before it is added (no contraction), as the other routes' host-side sums do.
__global__ void k_q_direct(int n, const double* __restrict__ s, const double* __restrict__ ct, double* q) {
  const int64_t L2 = 2 * ((int64_t)n + 1);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x + 1; k <= n; k += gridDim.x * blockDim.x) {
    double acc = s[0];
    int64_t ph = 0;
    for (int j = 1; j < n; ++j) {
      ph += k;
      if (ph >= L2) ph -= L2;
      acc = __dadd_rn(acc, __dmul_rn(2.0 * s[j], ct[ph]));
    }
    q[k - 1] = acc;
  }
}

cudaError_t launch_q_direct(int n, const double* s, const double* ct, double* q, cudaStream_t st) {
  const int blocks = (n + 127) / 128;
  k_q_direct<<<blocks < 4096 ? blocks : 4096, 128, 0, st>>>(n, s, ct, q);
  return cudaGetLastError();
}

}  // namespace tau
