// Element-type helpers (double, float, double-float), complex arithmetic and the in-place
// shared-memory FFTs of power-of-two length shared by the line passes (tau_kernels.cu) and the
// long-line route (tau_long.cu).
#pragma once

#include "tau_internal.cuh"

namespace tau {

// ---------------------------------------------------------------------------
// element-type helpers (double, float, double-float) and complex arithmetic
// ---------------------------------------------------------------------------
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }
// double-float product left as an unnormalised pair: the FMA-exact product of the high parts and
// the sum of its error with the two cross terms (|lo| within a few units in the last place of hi);
// a following double-float addition's two-sum absorbs it, so a multiply-add renormalises once
__device__ __forceinline__ df64 mul_pair(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df64{p, e};
}
__device__ __forceinline__ df64 tfma(df64 a, df64 b, df64 c) { return mul_pair(a, b) + c; }
__device__ __forceinline__ double shfl_up(double v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_up(float v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df64 shfl_up(df64 v, int o) {
  return df64{__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ double shfl_idx(double v, int s) { return __shfl_sync(0xffffffffu, v, s); }
__device__ __forceinline__ float shfl_idx(float v, int s) { return __shfl_sync(0xffffffffu, v, s); }
__device__ __forceinline__ df64 shfl_idx(df64 v, int s) {
  return df64{__shfl_sync(0xffffffffu, v.hi, s), __shfl_sync(0xffffffffu, v.lo, s)};
}
template <typename V> __device__ __forceinline__ V mk(decltype(V::x) x, decltype(V::x) y) { return V{x, y}; }
// read-only cached load for table entries (plain load for the double-float pair type)
template <typename V> __device__ __forceinline__ V ldt(const V* p) { return __ldg(p); }
template <> __device__ __forceinline__ df64x2 ldt<df64x2>(const df64x2* p) { return *p; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk<V>(tfma(a.x, b.x, -a.y * b.y), tfma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return mk<V>(tfma(a.x, b.x, a.y * b.y), tfma(a.y, b.x, -a.x * b.y));
}
// double-float complex products: each part the sum of two unnormalised products, one renormalisation
template <> __device__ __forceinline__ df64x2 cmul<df64x2>(df64x2 a, df64x2 b) {
  return df64x2{mul_pair(a.x, b.x) + (-mul_pair(a.y, b.y)), mul_pair(a.x, b.y) + mul_pair(a.y, b.x)};
}
template <> __device__ __forceinline__ df64x2 cmulc<df64x2>(df64x2 a, df64x2 b) {
  return df64x2{mul_pair(a.x, b.x) + mul_pair(a.y, b.y), mul_pair(a.y, b.x) + (-mul_pair(a.x, b.y))};
}
template <typename V> __device__ __forceinline__ V mul_mi(V a) { return mk<V>(a.y, -a.x); }  // -i a
template <typename V> __device__ __forceinline__ V mul_pi(V a) { return mk<V>(-a.y, a.x); }  // +i a

// Base-4 digit reversal of an nb-bit number (nb even): bit reversal, then a swap inside every
// pair of bits.
__device__ __forceinline__ int rev4(int x, int nb) {
  if (nb == 0) return 0;
  const unsigned r = __brev((unsigned)x) >> (32 - nb);
  return (int)(((r & 0x55555555u) << 1) | ((r >> 1) & 0x55555555u));
}

// Position of DFT output k after the in-place radix-4 (final radix-2 when log2 K is odd) DIF:
// the base-4 digits of k reversed; for odd log2 K the top bit of k is the last (radix-2) digit.
__device__ __forceinline__ int dif_pos(int k, int K) {
  const int lg = __ffs(K) - 1;
  if (lg & 1) {
    const int lo = lg - 1;
    return (rev4(k & ((1 << lo) - 1), lo) << 1) | (k >> lo);
  }
  return rev4(k, lg);
}

// Radix-4 decimation-in-frequency butterfly on registers (span q, index i within the group).
template <typename V>
__device__ __forceinline__ void dif4(V& a0, V& a1, V& a2, V& a3, int i, int q, const V* __restrict__ tws) {
  const V b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3), b3 = mul_mi(csub(a1, a3));
  a0 = cadd(b0, b2);
  if (i == 0) {
    a1 = cadd(b1, b3);
    a2 = csub(b0, b2);
    a3 = csub(b1, b3);
  } else {
    a1 = cmul(cadd(b1, b3), ldt(&tws[i]));
    a2 = cmul(csub(b0, b2), ldt(&tws[q + i]));
    a3 = cmul(csub(b1, b3), ldt(&tws[2 * q + i]));
  }
}

// The same butterfly when a2 = a3 = 0 (upper half of a zero-padded input, first stage only).
template <typename V>
__device__ __forceinline__ void dif4_lo(V& a0, V& a1, V& a2, V& a3, int i, int q, const V* __restrict__ tws) {
  const V b3 = mul_mi(a1);
  const V s0 = cadd(a0, a1), s1 = cadd(a0, b3), s2 = csub(a0, a1), s3 = csub(a0, b3);
  a0 = s0;
  if (i == 0) {
    a1 = s1;
    a2 = s2;
    a3 = s3;
  } else {
    a1 = cmul(s1, ldt(&tws[i]));
    a2 = cmul(s2, ldt(&tws[q + i]));
    a3 = cmul(s3, ldt(&tws[2 * q + i]));
  }
}

// a + w b and a - w b in six FMAs: the difference is formed as 2a - (a + w b).
template <typename V>
__device__ __forceinline__ void bfly2w(V& a, V& b, const V w) {
  using T = decltype(V::x);
  const T two = from_f<T>(2.0f);
  const T px = tfma(-w.y, b.y, tfma(w.x, b.x, a.x));
  const T py = tfma(w.y, b.x, tfma(w.x, b.y, a.y));
  b = mk<V>(tfma(two, a.x, -px), tfma(two, a.y, -py));
  a = mk<V>(px, py);
}
// a + w b only (four FMAs)
template <typename V>
__device__ __forceinline__ V bfly2w_sum(const V a, const V b, const V w) {
  return mk<V>(tfma(-w.y, b.y, tfma(w.x, b.x, a.x)), tfma(w.y, b.x, tfma(w.x, b.y, a.y)));
}

// Radix-4 decimation-in-time butterfly on registers, split as radix-2 x 2 so every twiddle
// multiply folds into the butterfly's additions (24 FMAs instead of 28 operations):
//   c = y0 +- w2 y2,  e = y1 +- w2 y3,  out0/2 = c0 +- w1 e0,  out1/3 = c1 +- (-+i w1) e1
// with w1 = w^i, w2 = w^2i (w = exp(-+2 pi i / size); INV conjugates).  Outputs land at offsets
// 0, q, 2q, 3q in y0, y1, y2, y3.  HALF computes out0 and out1 only.
template <bool INV, bool HALF, typename V>
__device__ __forceinline__ void dit4(V& y0, V& y1, V& y2, V& y3, int i, int q, const V* __restrict__ tws) {
  if (i == 0) {
    const V c0 = cadd(y0, y2), c1 = csub(y0, y2), e0 = cadd(y1, y3);
    const V e1 = INV ? mul_pi(csub(y1, y3)) : mul_mi(csub(y1, y3));
    y0 = cadd(c0, e0);
    y1 = cadd(c1, e1);
    if (!HALF) {
      y2 = csub(c0, e0);
      y3 = csub(c1, e1);
    }
    return;
  }
  V w1 = ldt(&tws[i]), w2 = ldt(&tws[q + i]);
  if (INV) {
    w1.y = -w1.y;
    w2.y = -w2.y;
  }
  // -i w1 (forward) or +i conj(w1) (inverse)
  const V wj = INV ? mk<V>(-w1.y, w1.x) : mk<V>(w1.y, -w1.x);
  bfly2w(y0, y2, w2);   // y0 = c0, y2 = c1
  bfly2w(y1, y3, w2);   // y1 = e0, y3 = e1
  if (HALF) {
    const V o0 = bfly2w_sum(y0, y1, w1);
    y1 = bfly2w_sum(y2, y3, wj);
    y0 = o0;
    return;
  }
  bfly2w(y0, y1, w1);   // y0 = out0, y1 = out2
  bfly2w(y2, y3, wj);   // y2 = out1, y3 = out3
  const V o2 = y1;
  y1 = y2;
  y2 = o2;
}

// Forward complex DFT of length K (natural order in, digit-reversed out) on nl lines stored at
// cb + l*cs, twiddles from the stage-packed table twp (twp_size(K) entries).  Each thread loads two
// independent butterflies before computing either, so their shared-memory latencies overlap.
// zero_hi: entries [K/2, K) are zero and not read (the first stage skips them).  stop_last: the
// last stage (size 4, or 2 for odd log2 K) is left to the caller (toep_mid).
// Caller synchronises before; this synchronises after.
template <typename V>
__device__ void fft_dif(V* cb, int cs, int nl, int K, const V* __restrict__ twp, bool zero_hi = false,
                        bool stop_last = false) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int lgK = __ffs(K) - 1;
  const int min_r4 = (stop_last && !(lgK & 1)) ? 16 : 4;
  int size = K, lgs = lgK;
  for (; size >= min_r4; size >>= 2, lgs -= 2) {
    const int q = size >> 2, lq = lgs - 2, lnb = lgK - 2;
    const V* __restrict__ tws = twp + (K - size);
    const int nb = K >> 2;
    const int tot = nl * nb;
    for (int b = tid; b < tot; b += 2 * T) {
      const int bb = b + T;
      const bool two = bb < tot;
      int l = b >> lnb, loc = b & (nb - 1);
      int g = loc >> lq;
      const int i0 = loc & (q - 1);
      V* x = cb + l * cs + (g << lgs) + i0;
      int i1 = 0;
      V* y = x;
      if (two) {
        l = bb >> lnb;
        loc = bb & (nb - 1);
        g = loc >> lq;
        i1 = loc & (q - 1);
        y = cb + l * cs + (g << lgs) + i1;
      }
      if (zero_hi && size == K) {
        V a0 = x[0], a1 = x[q], a2, a3;
        V c0, c1, c2, c3;
        if (two) {
          c0 = y[0];
          c1 = y[q];
        }
        dif4_lo(a0, a1, a2, a3, i0, q, tws);
        if (two) dif4_lo(c0, c1, c2, c3, i1, q, tws);
        x[0] = a0;
        x[q] = a1;
        x[2 * q] = a2;
        x[3 * q] = a3;
        if (two) {
          y[0] = c0;
          y[q] = c1;
          y[2 * q] = c2;
          y[3 * q] = c3;
        }
        continue;
      }
      V a0 = x[0], a1 = x[q], a2 = x[2 * q], a3 = x[3 * q];
      V c0, c1, c2, c3;
      if (two) {
        c0 = y[0];
        c1 = y[q];
        c2 = y[2 * q];
        c3 = y[3 * q];
      }
      dif4(a0, a1, a2, a3, i0, q, tws);
      if (two) dif4(c0, c1, c2, c3, i1, q, tws);
      x[0] = a0;
      x[q] = a1;
      x[2 * q] = a2;
      x[3 * q] = a3;
      if (two) {
        y[0] = c0;
        y[q] = c1;
        y[2 * q] = c2;
        y[3 * q] = c3;
      }
    }
    __syncthreads();
  }
  if (size == 2 && !stop_last) {
    const int nb = K >> 1;
    for (int b = tid; b < nl * nb; b += T) {
      const int l = b >> (lgK - 1), loc = b & (nb - 1);
      V* x = cb + l * cs + 2 * loc;
      const V a0 = x[0], a1 = x[1];
      x[0] = cadd(a0, a1);
      x[1] = csub(a0, a1);
    }
    __syncthreads();
  }
}

// Complex DFT of length K by decimation in time: digit-reversed in (the order fft_dif leaves and
// dif_pos() describes), natural order out, same twiddle table as fft_dif.  INV: the unnormalised
// inverse (times K).  half_out: only outputs [0, K/2) are needed (the last stage skips the rest).
// skip_first: the first stage (size 4, or 2 for odd log2 K) was done by the caller (toep_mid).
template <bool INV, typename V>
__device__ void fft_dit(V* cb, int cs, int nl, int K, const V* __restrict__ twp, bool half_out = false,
                        bool skip_first = false) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int lgK = __ffs(K) - 1;
  int size = 4, lgs = 2;
  if (skip_first && !(lgK & 1)) {
    size = 16;
    lgs = 4;
  }
  if ((lgK & 1) && skip_first) {
    size = 8;
    lgs = 3;
  } else if (lgK & 1) {
    const int nb = K >> 1;
    for (int b = tid; b < nl * nb; b += T) {
      const int l = b >> (lgK - 1), loc = b & (nb - 1);
      V* x = cb + l * cs + 2 * loc;
      const V a0 = x[0], a1 = x[1];
      x[0] = cadd(a0, a1);
      x[1] = csub(a0, a1);
    }
    __syncthreads();
    size = 8;
    lgs = 3;
  }
  for (; size <= K; size <<= 2, lgs += 2) {
    const int q = size >> 2, lq = lgs - 2, lnb = lgK - 2;
    const V* __restrict__ tws = twp + (K - size);
    const int nb = K >> 2;
    const int tot = nl * nb;
    const bool half = half_out && size == K;
    for (int b = tid; b < tot; b += 2 * T) {
      const int bb = b + T;
      const bool two = bb < tot;
      int l = b >> lnb, loc = b & (nb - 1);
      int g = loc >> lq;
      const int i0 = loc & (q - 1);
      V* x = cb + l * cs + (g << lgs) + i0;
      int i1 = 0;
      V* y = x;
      if (two) {
        l = bb >> lnb;
        loc = bb & (nb - 1);
        g = loc >> lq;
        i1 = loc & (q - 1);
        y = cb + l * cs + (g << lgs) + i1;
      }
      V a0 = x[0], a1 = x[q], a2 = x[2 * q], a3 = x[3 * q];
      V c0, c1, c2, c3;
      if (two) {
        c0 = y[0];
        c1 = y[q];
        c2 = y[2 * q];
        c3 = y[3 * q];
      }
      if (half) {
        dit4<INV, true>(a0, a1, a2, a3, i0, q, tws);
        if (two) dit4<INV, true>(c0, c1, c2, c3, i1, q, tws);
        x[0] = a0;
        x[q] = a1;
        if (two) {
          y[0] = c0;
          y[q] = c1;
        }
        continue;
      }
      dit4<INV, false>(a0, a1, a2, a3, i0, q, tws);
      if (two) dit4<INV, false>(c0, c1, c2, c3, i1, q, tws);
      x[0] = a0;
      x[q] = a1;
      x[2 * q] = a2;
      x[3 * q] = a3;
      if (two) {
        y[0] = c0;
        y[q] = c1;
        y[2 * q] = c2;
        y[3 * q] = c3;
      }
    }
    __syncthreads();
  }
}

}  // namespace tau
