// CUDA kernels of the τ-preconditioned GMRES solver (sm_103a; FP64, with FP32 and double-float
// instantiations of the line passes and Gram-Schmidt kernels for the other precisions).
//
// Line passes: the matvec A x = B_alpha (e∘x) + sum_i eta_i (⊗_{l!=i} B_l ⊗ S_i) x of Eq. (tls),
// the right-hand side of Eq. (tls) and the DST-I based τ solve of Eqs. (Pa), (diag) are applied
// one dimension at a time.  A pass loads a tile of grid lines along one dimension into shared
// memory, works on them there and writes them back.  Two channels carry the Kronecker terms
// between passes: after the pass over dimension i,
//     a = (B_i ... B_1)(e∘x) + sum_{l<=i} eta_l (B_i..S_l..B_1) x,      c = (B_i ... B_1) x,
// so the pass over dimension i+1 computes a' = B_{i+1} a + eta_{i+1} S_{i+1} c, c' = B_{i+1} c.
//
// FFT route (n_i + 1 = K = 2^p): the Toeplitz product S_i x uses the circulant embedding of length
// 2K, whose real transforms run as one complex FFT of length K in place in the padded line (radix-4
// decimation in frequency, digit-reversed output located by dif_pos(); the spectral step works in
// that layout; the inverse is the mirrored decimation in time, so no reordering pass is needed).
// The DST-I of length n_i is a real FFT of length K: a complex FFT of length K/2 (decimation in time
// fed by a digit-reversed scatter), a pair recombination and a prefix sum.  Dense route (any n_i):
// explicit O(n_i) sums per output.
#include "tau_internal.cuh"
#include "tau_fft.cuh"
#include "tau_group.cuh"

#include <math.h>

#include <type_traits>

namespace tau {

thread_local std::vector<LaunchRec>* tl_rec = nullptr;

constexpr int PASS_THREADS = 128;       // threads of a line-pass CTA (the wide variant: 256)
constexpr int PASS_MAX_THREADS = 256;


// FP64 route of the spectral step: one pass over the pairs (k, K-k) in the digit-reversed layout
// (the fused toep_mid below raises the FP64 kernel's register pressure more than it saves).
template <typename V>
__device__ __forceinline__ void toep_pair(V* x, int k, int K, const V* __restrict__ spec) {
  const int kk = (K - k) & (K - 1);
  const int pk = dif_pos(k, K), pkk = dif_pos(kk, K);
  const V A = x[pk], B = x[pkk];
  const V ca = ldt(&spec[4 * k]), cbv = ldt(&spec[4 * k + 1]);
  x[pk] = mk<V>(tfma(ca.x, A.x, tfma(-ca.y, A.y, tfma(cbv.x, B.x, cbv.y * B.y))),
                tfma(ca.x, A.y, tfma(ca.y, A.x, tfma(cbv.y, B.x, -cbv.x * B.y))));
  if (kk != k) {
    const V cc = ldt(&spec[4 * k + 2]), cd = ldt(&spec[4 * k + 3]);
    x[pkk] = mk<V>(tfma(cc.x, A.x, tfma(cc.y, A.y, tfma(cd.x, B.x, -cd.y * B.y))),
                   tfma(cc.y, A.x, tfma(-cc.x, A.y, tfma(cd.x, B.y, cd.y * B.x))));
  }
}

template <typename V>
__device__ void toep_spectral(V* cb, int cs, int nl, int K, const V* __restrict__ spec) {
  const int T = blockDim.x, tid = threadIdx.x;
  // slot k in [0, K/2) of each line: the pair (k, K-k); slot 0 also takes the pair (K/2, K/2)
  const int H = K > 1 ? K >> 1 : 1, lh = __ffs(H) - 1;
  for (int b = tid; b < (nl << lh); b += T) {
    const int l = b >> lh, k = b & (H - 1);
    V* x = cb + l * cs;
    toep_pair(x, k, K, spec);
    if (k == 0 && K > 1) toep_pair(x, K >> 1, K, spec);
  }
  __syncthreads();
}

// Spectral step of the Toeplitz product: multiply the length-2K real DFT of the packed sequence by
// the real symmetric circulant spectrum, working on the packed half-length DFT Z.  For each pair
// (k, K-k) the step is the linear map
//   Z'_k = a_k Z_k + b_k conj(Z_{K-k}),   Z'_{K-k} = c_k conj(Z_k) + d_k Z_{K-k}
// whose coefficients spec[4k..4k+3] = (a, b, c, d) fold the unpacking (E = Z_k + conj Z_{K-k},
// O = -i (Z_k - conj Z_{K-k}), Y_k = (E + W_k O)/2, W_k = exp(-i pi k/K)), the multiply by lambda
// and the repacking, scaled by 1/K for the unnormalised inverse (toep_pack_coeffs).
// One pair in registers: A = Z_k, B = Z_{K-k}, k <= K/2; a self-paired k (0 or K/2) updates A alone.
template <typename V>
__device__ __forceinline__ void spec_apply(V& A, V& B, int k, bool self, const V* __restrict__ spec) {
  const V ca = ldt(&spec[4 * k]), cbv = ldt(&spec[4 * k + 1]);
  const V Bv = self ? A : B;
  const V nA = mk<V>(tfma(ca.x, A.x, tfma(-ca.y, A.y, tfma(cbv.x, Bv.x, cbv.y * Bv.y))),
                     tfma(ca.x, A.y, tfma(ca.y, A.x, tfma(cbv.y, Bv.x, -cbv.x * Bv.y))));
  if (!self) {
    const V cc = ldt(&spec[4 * k + 2]), cd = ldt(&spec[4 * k + 3]);
    B = mk<V>(tfma(cc.x, A.x, tfma(cc.y, A.y, tfma(cd.x, B.x, -cd.y * B.y))),
              tfma(cc.y, A.x, tfma(-cc.x, A.y, tfma(cd.x, B.y, cd.y * B.x))));
  }
  A = nA;
}

// u holds Z_{k1}, w holds Z_{K-k1}: apply the pair's map whichever of the two has the lower index.
template <typename V>
__device__ __forceinline__ void spec_pairup(V& u, V& w, int k1, int K, const V* __restrict__ spec) {
  const int k2 = (K - k1) & (K - 1);
  if (k1 == k2) spec_apply(u, u, k1, true, spec);
  else if (k1 < k2) spec_apply(u, w, k1, false, spec);
  else spec_apply(w, u, k2, false, spec);
}

// The forward DIF's last stage, the spectral map and the inverse DIT's first stage in one pass.
// The last DIF stage (radix R = 4, or 2 for odd log2 K; no twiddles) leaves in the R consecutive
// slots of group g the frequencies k_lo + r K/R, r < R, with g the digit reversal of k_lo; the
// partners K - k of a group's frequencies fill group g' = rev(K/R - k_lo) in reversed slot order.
// One thread takes both groups from shared memory (two contiguous runs, no bank conflicts),
// finishes the forward transform, applies the R 2x2 maps and starts the inverse transform.
template <typename V>
__device__ __forceinline__ void toep_mid_r4(V* x, int klo, int lgG, int K, const V* __restrict__ spec) {
  const int G = 1 << lgG;
  const int g = rev4(klo, lgG), g2 = rev4((G - klo) & (G - 1), lgG);
  const V* __restrict__ none = nullptr;
  V a0 = x[4 * g], a1 = x[4 * g + 1], a2 = x[4 * g + 2], a3 = x[4 * g + 3];
  dif4(a0, a1, a2, a3, 0, 1, none);
  if (g2 != g) {
    V b0 = x[4 * g2], b1 = x[4 * g2 + 1], b2 = x[4 * g2 + 2], b3 = x[4 * g2 + 3];
    dif4(b0, b1, b2, b3, 0, 1, none);
    spec_pairup(a0, b3, klo, K, spec);
    spec_pairup(a1, b2, klo + G, K, spec);
    spec_pairup(a2, b1, klo + 2 * G, K, spec);
    spec_pairup(a3, b0, klo + 3 * G, K, spec);
    dit4<true, false>(b0, b1, b2, b3, 0, 1, none);
    x[4 * g2] = b0;
    x[4 * g2 + 1] = b1;
    x[4 * g2 + 2] = b2;
    x[4 * g2 + 3] = b3;
  } else if (klo == 0) {
    spec_pairup(a0, a0, 0, K, spec);
    spec_pairup(a2, a2, 2 * G, K, spec);
    spec_pairup(a1, a3, G, K, spec);
  } else {  // klo = G/2: the group pairs with itself, slot r with slot 3 - r
    spec_pairup(a0, a3, klo, K, spec);
    spec_pairup(a1, a2, klo + G, K, spec);
  }
  dit4<true, false>(a0, a1, a2, a3, 0, 1, none);
  x[4 * g] = a0;
  x[4 * g + 1] = a1;
  x[4 * g + 2] = a2;
  x[4 * g + 3] = a3;
}

template <typename V>
__device__ __forceinline__ void toep_mid_r2(V* x, int klo, int lgG, int K, const V* __restrict__ spec) {
  const int G = 1 << lgG;
  const int g = rev4(klo, lgG), g2 = rev4((G - klo) & (G - 1), lgG);
  const V p0 = x[2 * g], p1 = x[2 * g + 1];
  V a0 = cadd(p0, p1), a1 = csub(p0, p1);
  if (g2 != g) {
    const V q0 = x[2 * g2], q1 = x[2 * g2 + 1];
    V b0 = cadd(q0, q1), b1 = csub(q0, q1);
    spec_pairup(a0, b1, klo, K, spec);
    spec_pairup(a1, b0, klo + G, K, spec);
    x[2 * g2] = cadd(b0, b1);
    x[2 * g2 + 1] = csub(b0, b1);
  } else if (klo == 0) {
    spec_pairup(a0, a0, 0, K, spec);
    spec_pairup(a1, a1, G, K, spec);
  } else {  // klo = G/2
    spec_pairup(a0, a1, klo, K, spec);
  }
  x[2 * g] = cadd(a0, a1);
  x[2 * g + 1] = csub(a0, a1);
}

// The forward DIF's last stage, the spectral map and the inverse DIT's first stage in one pass.
// The last DIF stage (radix R = 4, or 2 for odd log2 K; no twiddles) leaves in the R consecutive
// slots of group g the frequencies k_lo + r K/R, r < R, with g the digit reversal of k_lo; the
// partners K - k of a group's frequencies fill group g' = rev(K/R - k_lo) in reversed slot order.
// Work item k_lo in [0, G/2] (G = K/R) takes both groups from shared memory (two contiguous runs),
// finishes the forward transform, applies the R 2x2 maps and starts the inverse transform; item
// slot 0 also takes the self-paired k_lo = G/2, so every lane has work.
template <typename V>
__device__ void toep_mid(V* cb, int cs, int nl, int K, const V* __restrict__ spec) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int lgK = __ffs(K) - 1;
  const int lgG = (lgK & 1) ? lgK - 1 : lgK - 2, G = 1 << lgG;
  const int H = G > 1 ? G >> 1 : 1, lh = __ffs(H) - 1;
  for (int t = tid; t < (nl << lh); t += T) {
    const int l = t >> lh, klo = t & (H - 1);
    V* x = cb + l * cs;
    const int items = (klo == 0 && G > 1) ? 2 : 1;
#pragma unroll 1
    for (int it = 0; it < items; ++it) {
      const int kl = it ? G >> 1 : klo;
      if (lgK & 1) toep_mid_r2(x, kl, lgG, K, spec);
      else toep_mid_r4(x, kl, lgG, K, spec);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// tile geometry
// ---------------------------------------------------------------------------
struct TileGeo {
  int64_t base;   // address of element (l=0, j=0)
  int64_t lstep;  // address step between lines of the tile
  int64_t jstep;  // address step along a line
  int nvalid;     // number of valid lines in the tile
};

template <typename PT>
__device__ __forceinline__ TileGeo tile_geo(const PT& P, int64_t tile) {
  TileGeo t;
  const int64_t N = P.len;
  if (P.ax == 0) {
    const int64_t l0 = tile * P.lpb;
    t.base = l0 * N;
    t.lstep = N;
    t.jstep = 1;
    const int64_t rem = P.nlines - l0;
    t.nvalid = (int)(rem < P.lpb ? rem : P.lpb);
  } else {
    const int64_t tpo = (P.inner + P.lpb - 1) / P.lpb;
    const int64_t o = tile / tpo;
    const int64_t c0 = (tile - o * tpo) * P.lpb;
    t.base = o * N * P.inner + c0;
    t.lstep = 1;
    t.jstep = P.inner;
    const int64_t rem = P.inner - c0;
    t.nvalid = (int)(rem < P.lpb ? rem : P.lpb);
  }
  return t;
}

// Flat thread index -> (line l, position j) inside a tile.  Lines along x_1 (jstep 1): slots of
// 2^lgnp >= N per line (consecutive threads walk a line; slots j >= N are idle).  Lines along a
// strided dimension: consecutive threads take consecutive lines (lpb is a power of two).
__device__ __forceinline__ int tile_total(const TileGeo& t, int N, int lpb, int lgnp) {
  return t.jstep == 1 ? (lpb << lgnp) : N * lpb;
}
__device__ __forceinline__ bool tile_lj(const TileGeo& t, int N, int lpb, int lgnp, int idx, int& l, int& j) {
  if (t.jstep == 1) {
    l = idx >> lgnp;
    j = idx & ((1 << lgnp) - 1);
    return j < N;
  }
  const int llpb = __ffs(lpb) - 1;
  j = idx >> llpb;
  l = idx & (lpb - 1);
  return true;
}
__device__ __forceinline__ int lg_pad(int N) { return N > 1 ? 32 - __clz(N - 1) : 0; }

// sm[l*ss + j] = g[base + l*lstep + j*jstep]; consecutive threads take consecutive addresses.
// Each thread issues a batch of independent loads (8 of 4 bytes, 4 of 8) before the shared-memory
// stores, so one memory latency covers the batch instead of one per element.
template <typename S, typename T>
__device__ __forceinline__ void tile_load(const TileGeo& t, int N, int lpb, const S* __restrict__ g, T* sm, int ss) {
  constexpr int TILE_BATCH = sizeof(S) >= 8 ? 4 : 8;
  const int lgnp = lg_pad(N), tot = tile_total(t, N, lpb, lgnp);
  const int TH = blockDim.x;
  for (int base = threadIdx.x; base < tot; base += TILE_BATCH * TH) {
    S v[TILE_BATCH];
    int dst[TILE_BATCH];
#pragma unroll
    for (int r = 0; r < TILE_BATCH; ++r) {
      const int idx = base + r * TH;
      int l = 0, j = 0;
      dst[r] = -1;
      if (idx < tot && tile_lj(t, N, lpb, lgnp, idx, l, j)) {
        dst[r] = l * ss + j;
        v[r] = (l < t.nvalid) ? g[t.base + l * t.lstep + (int64_t)j * t.jstep] : from_f<S>(0.0f);
      }
    }
#pragma unroll
    for (int r = 0; r < TILE_BATCH; ++r)
      if (dst[r] >= 0) sm[dst[r]] = cvt<T, S>(v[r]);
  }
}

template <typename T>
__device__ __forceinline__ void tile_store(const TileGeo& t, int N, int lpb, const T* sm, int ss, T* g) {
  const int lgnp = lg_pad(N), tot = tile_total(t, N, lpb, lgnp);
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    int l, j;
    if (!tile_lj(t, N, lpb, lgnp, idx, l, j)) continue;
    if (l < t.nvalid) g[t.base + l * t.lstep + (int64_t)j * t.jstep] = sm[l * ss + j];
  }
}

// B_{alpha} along the line (3-point stencil of 𝓗_alpha, zero beyond the interior).
template <typename T>
__device__ __forceinline__ T stencil_B(const T* row, int j, int N, T bd, T bo) {
  const T lft = j > 0 ? row[j - 1] : from_f<T>(0.0f);
  const T rgt = j + 1 < N ? row[j + 1] : from_f<T>(0.0f);
  return tfma(bd, row[j], bo * (lft + rgt));
}

// ---------------------------------------------------------------------------
// per-line transforms on shared memory
// ---------------------------------------------------------------------------
// Dense-route transforms read the whole line for every output: they write their outputs to the
// second half of each row (row stride 2N) and this copies them back over the input after a barrier.
template <typename T>
__device__ __forceinline__ void dense_copy_back(T* xs, int xst, int lpb, int N) {
  __syncthreads();
  for (int idx = threadIdx.x; idx < lpb * N; idx += blockDim.x) {
    const int l = idx / N;
    xs[l * xst + idx - l * N] = xs[l * xst + N + idx - l * N];
  }
  __syncthreads();
}
// Toeplitz product T x in place for every line: x_j at xs[l*xst + j].  FFT route: xst = 2K and
// the line's 2K reals are the packed complex sequence z_j = (y_2j, y_2j+1) of the zero-padded
// y (y_t = x_t for t < N, 0 otherwise), so packing is only y_N = 0 (the upper half is zero by
// construction and skipped) and the product comes back in [0, N).  Chirp route: the same with K the
// power of two >= N + 1 and xst >= 2K.  Dense route: xst = N.
template <typename T>
__device__ void toeplitz_lines(const PassT<T>& P, T* xs, int xst) {
  using V = vec2<T>;
  const int N = P.len, lpb = P.lpb;
  const int TH = blockDim.x, tid = threadIdx.x;
  if (P.dim.route != ROUTE_DENSE) {
    const int K = P.dim.K;
    // y_t = 0 for t in [N, K) (one slot on the FFT route, where K = N + 1); z_j for j >= K/2 is
    // zero and never read when the first DIF
    // stage skips it (K >= 4, or K > 4 where the last DIF stage is fused into toep_mid).
    constexpr bool fused = !std::is_same<T, double>::value;
    const int zn = (fused ? K > 4 : K >= 4) ? K - N : 2 * K - N;
    for (int b = tid; b < lpb * zn; b += TH) {
      const int l = b / zn;
      xs[l * xst + N + (b - l * zn)] = from_f<T>(0.0f);
    }
    __syncthreads();
    // line l's packed sequence starts at xs + l*xst (xst = 2K on the FFT route; on the chirp route
    // the row is longer than the 2K reals the product uses)
    V* cb = reinterpret_cast<V*>(xs);
    const int cs = xst >> 1;
    // outputs y_t, t < N, are z_j for j < K/2 (half_out of the inverse's last stage)
    if constexpr (fused) {
      fft_dif(cb, cs, lpb, K, P.dim.twK, K > 4, true);
      toep_mid(cb, cs, lpb, K, P.dim.spec);
      fft_dit<true>(cb, cs, lpb, K, P.dim.twK, true, true);
    } else {
      fft_dif(cb, cs, lpb, K, P.dim.twK, K >= 4);
      toep_spectral(cb, cs, lpb, K, P.dim.spec);
      fft_dit<true>(cb, cs, lpb, K, P.dim.twK, true);
    }
  } else {
    // dense: (T x)_a = sum_b s_|a-b| x_b.  Every output reads the whole line, so the outputs go to
    // the second half of the row (xst = 2N) and are copied back once all of them are computed.
    const T* __restrict__ s = P.dim.s;
    const T z0 = from_f<T>(0.0f);
    const int tot = lpb * N;
    for (int idx = tid; idx < tot; idx += TH) {
      const int l = idx / N, a = idx - l * N;
      const T* row = xs + l * xst;
      T sacc = z0;
      for (int bb = 0; bb < N; ++bb) sacc = tfma(s[abs(a - bb)], row[bb], sacc);
      xs[l * xst + N + a] = sacc;
    }
    dense_copy_back(xs, xst, lpb, N);
  }
}

// Orthonormal Hartley transform of every line in place (dense, any n): y_k = sum_j c_{jk mod n} x_j
// with c_t = cas(2 pi t / n) / sqrt(n), x_j at xs[l*xst + j], j, k = 0..n-1.  It is its own inverse and
// diagonalises the Strang circulants of the comparison preconditioner P_c (their spectra are even).
template <typename T>
__device__ void hartley_lines(const PassT<T>& P, T* xs, int xst) {
  const int N = P.len, lpb = P.lpb;
  const int TH = blockDim.x, tid = threadIdx.x;
  const T* __restrict__ ct = P.dim.cas;
  const T z0 = from_f<T>(0.0f);
  const int tot = lpb * N;
  for (int idx = tid; idx < tot; idx += TH) {
    const int l = idx / N, k = idx - l * N;
    const T* row = xs + l * xst;
    T sacc = z0;
    int ph = 0;  // (j * k) mod N
    for (int j = 0; j < N; ++j) {
      sacc = tfma(ct[ph], row[j], sacc);
      ph += k;
      if (ph >= N) ph -= N;
    }
    xs[l * xst + N + k] = sacc;
  }
  dense_copy_back(xs, xst, lpb, N);
}

// Prefix sums over the even slots of each line of the DST recombination:
//   row[2k] <- sum_{i<=k} row[2i] - row[0]/2,  k < K2,
// which turns the stored sc Re W_k into the odd outputs y_{2k+1}.  row[0] itself is left unchanged
// by any partial scan, so it can be read until the final pass writes it.
//
// FP64: each thread scans a contiguous segment of K2 / spl slots sequentially (one addition per
// slot; FP64 additions are the scarce resource), segment offsets by a block-wide shuffle scan.
template <typename T>
__device__ void prefix_segments(T* xs, int xst, int lpb, int K2) {
  const int TH = blockDim.x, tid = threadIdx.x;
  __shared__ T scan_incl[PASS_MAX_THREADS];
  __shared__ T warp_tot[PASS_MAX_THREADS / 32];
  int spl = TH / lpb;
  if (spl < 1) spl = 1;
  spl = 1 << (31 - __clz(spl));
  if (spl > K2) spl = K2;
  const int lspl = __ffs(spl) - 1;
  const int seg = K2 >> lspl;
  const int l = tid >> lspl, sg = tid & (spl - 1);
  const bool act = l < lpb;
  T* row = xs + (act ? l : 0) * xst;
  T acc = from_f<T>(0.0f);
  if (act) {
    for (int k = sg * seg; k < (sg + 1) * seg; ++k) {
      acc += row[2 * k];
      row[2 * k] = acc;
    }
  }
  const int lane = tid & 31, wp = tid >> 5;
  T v = acc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T t = shfl_up(v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_tot[wp] = v;
  __syncthreads();
  // read before the barrier that precedes the offset loop, the only writer of row[0]
  const T half0 = from_f<T>(0.5f) * row[0];
  for (int w2 = 0; w2 < wp; ++w2) v += warp_tot[w2];
  scan_incl[tid] = v;
  __syncthreads();
  if (act) {
    const T base = l * spl > 0 ? scan_incl[l * spl - 1] : from_f<T>(0.0f);
    const T off = v - acc - base - half0;
    for (int k = sg * seg; k < (sg + 1) * seg; ++k) row[2 * k] += off;
  }
  __syncthreads();
}

// FP32 pipes (float, double-float): warps scan 32 consecutive slots at a time with shuffles and a
// running carry, so consecutive lanes touch consecutive slots (no bank conflicts) and a line owned
// by one warp needs no block barrier.  A line shared by wpl > 1 warps (fewer lines than warps) is
// split into wpl portions whose totals are combined through shared memory.
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T t = shfl_up(v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <typename T>
__device__ void prefix_warps(T* xs, int xst, int lpb, int K2) {
  const int NW = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T half = from_f<T>(0.5f), z0 = from_f<T>(0.0f);
  int wpl = lpb >= NW ? 1 : NW / lpb;
  if (K2 < 32 * wpl) wpl = 1;
  if (wpl == 1) {
    for (int l = wid; l < lpb; l += NW) {
      T* row = xs + l * xst;
      const T h0 = half * row[0];
      T carry = z0;
      for (int c = 0; c < K2; c += 32) {
        const int k = c + lane;
        T v = k < K2 ? row[2 * k] : z0;
        v = warp_incl_scan(v, lane) + carry;
        if (k < K2) row[2 * k] = v - h0;
        carry = shfl_idx(v, 31);
      }
    }
    __syncthreads();
    return;
  }
  __shared__ T part_tot[PASS_MAX_THREADS / 32];
  const int l = wid / wpl, pw = wid - l * wpl;
  const int part = K2 / wpl, k0 = pw * part;
  T* row = xs + l * xst;
  T carry = z0;
  for (int c = 0; c < part; c += 32) {
    const int k = k0 + c + lane;
    const T v = warp_incl_scan(row[2 * k], lane) + carry;
    if (k != 0) row[2 * k] = v;   // the prefix at slot 0 is row[0] itself
    carry = shfl_idx(v, 31);
  }
  if (lane == 0) part_tot[wid] = carry;
  const T h0 = half * row[0];   // no warp writes row[0] before the barrier below
  __syncthreads();
  T off = -h0;
  for (int q = l * wpl; q < wid; ++q) off += part_tot[q];
  for (int c = 0; c < part; c += 32) row[2 * (k0 + c + lane)] += off;
  __syncthreads();
}

// Packed input z_m = (w_2m, w_2m+1) of the DST's half-length FFT (FP32 fused input stage):
// w_j = sn_j (x_j + x_{K-j}) + hh (x_j - x_{K-j}), w_0 = 0, x_j at row[j-1].
__device__ __forceinline__ float2 dst_packed_input(const float* row, int m, int K, const float* __restrict__ sn,
                                                   float hh) {
  float w[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = 2 * m + r;
    float v = 0.0f;
    if (j > 0) {
      const float xj = row[j - 1], xk = row[K - j - 1];
      v = fmaf(sn[j], xj + xk, hh * (xj - xk));
    }
    w[r] = v;
  }
  return make_float2(w[0], w[1]);
}

// Chirp route DST-I of every line in place, two lines per convolution.  As on the FFT route the
// DST-I of a line is a real DFT of length L = n + 1 of w_j = sin(pi j/L)(x_j + x_{L-j}) +
// (x_j - x_{L-j})/2 (x_0 = x_L = 0): y_{2k} = -Im W_k, y_{2k+1} - y_{2k-1} = Re W_k, y_1 = Re W_0/2
// (scaled by sqrt(2/L)).  Lines a, b of a pair share one complex DFT of v = w^a + i w^b, taken by
// Bluestein's method: with c_m = exp(-i pi m^2/L), V_k = c_k sum_j (v_j c_j) conj(c_{k-j}) (v_0 = 0,
// so the lags k - j span [-n, n-1]), a circular convolution of power-of-two length M >= 2n run as
// forward DIF (upper half zero), product with the kernel's spectrum bhat (digit-reversed order of
// the DIF, scaled by sqrt(2/L)/(2M)) and inverse DIT.  When M >= 2L, v_j sits at j and the inverse
// computes its first half only; when M = 2n (n a power of two) v_j sits at j - 1, inside the half
// the first DIF stage reads, and the inverse runs in full (z_0 lands at M - 1).  Then
// W^a_k = V_k + conj V_{L-k}, W^b_k = -i (V_k - conj V_{L-k}) (V_L = V_0); the prefix sum gives
// the odd outputs.
// Layout: rows of xst = 2K reals (an even number of them: an odd last line pairs with a zero line);
// the pair buffer of lines 2p, 2p+1 is their two rows (2K complex).  The lines are first copied to
// scr (n reals per line), which also takes the recombined outputs before they return to the rows.
template <typename T>
__device__ void dst_chirp_lines(const PassT<T>& P, T* xs, int xst, T* scr) {
  using V = vec2<T>;
  const int N = P.len, lpb = P.lpb, M = P.dim.M, L = N + 1, K = P.dim.K;
  const int TH = blockDim.x, tid = threadIdx.x;
  const int npair = (lpb + 1) >> 1;
  const V* __restrict__ c = P.dim.chirp;
  const V* __restrict__ bh = P.dim.bhat;
  const T* __restrict__ sn = P.dim.sintab;   // sin(pi t / L)
  const T z0 = from_f<T>(0.0f), half = from_f<T>(0.5f);
  V* cb = reinterpret_cast<V*>(xs);           // pair p at cb + p*xst (complex)
  for (int b = tid; b < lpb * N; b += TH) {
    const int l = b / N;
    scr[b] = xs[l * xst + (b - l * N)];
  }
  __syncthreads();
  // v_j c_j at position j - sh for 1 <= j < L; zero elsewhere up to M/2 (the whole line when M <= 4,
  // where the first DIF stage reads it)
  const int sh = M < 2 * L ? 1 : 0;
  const int fill = M > 4 ? M >> 1 : M, lgf = __ffs(fill) - 1;
  for (int b = tid; b < (npair << lgf); b += TH) {
    const int pr = b >> lgf, pos = b & (fill - 1), j = pos + sh;
    V v = mk<V>(z0, z0);
    if (j > 0 && j < L) {
      const T s = sn[j];
      T w[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int l = 2 * pr + r;
        w[r] = z0;
        if (l < lpb) {
          const T xj = scr[l * N + j - 1], xk = scr[l * N + L - j - 1];
          w[r] = tfma(s, xj + xk, half * (xj - xk));
        }
      }
      v = cmul(mk<V>(w[0], w[1]), ldt(&c[j]));
    }
    cb[pr * xst + pos] = v;
  }
  __syncthreads();
  const int lgM = __ffs(M) - 1;
  fft_dif(cb, xst, npair, M, P.dim.twM, M > 4);
  for (int b = tid; b < (npair << lgM); b += TH) {
    const int pr = b >> lgM, pos = b & (M - 1);
    V* x = cb + pr * xst + pos;
    *x = cmul(*x, ldt(&bh[pos]));
  }
  __syncthreads();
  fft_dit<true>(cb, xst, npair, M, P.dim.twM, M > 4 && !sh);
  // recombination, k = 0..N/2 (z_k at position (k - sh) mod M): Re W_k to scr[2k] (odd outputs, before the prefix sum), -Im W_k =
  // y_{2k} to scr[2k-1]
  const int nk = N / 2 + 1;
  for (int b = tid; b < npair * nk; b += TH) {
    const int pr = b / nk, k = b - pr * nk, km = k ? L - k : 0;
    const V vk = cmul(ldt(&c[k]), cb[pr * xst + ((k - sh) & (M - 1))]);
    const V vm = cmul(ldt(&c[km]), cb[pr * xst + ((km - sh) & (M - 1))]);
    const V wa = mk<V>(vk.x + vm.x, vk.y - vm.y);
    const V wb = mk<V>(vk.y + vm.y, vm.x - vk.x);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int l = 2 * pr + r;
      if (l >= lpb) continue;
      const V W = r ? wb : wa;
      if (2 * k < N) scr[l * N + 2 * k] = W.x;
      if (k >= 1) scr[l * N + 2 * k - 1] = -W.y;
    }
  }
  __syncthreads();
  // back to the rows, zero from n to K (the prefix sum runs over the K/2 even slots below K)
  const int lgK = __ffs(K) - 1;
  for (int b = tid; b < (lpb << lgK); b += TH) {
    const int l = b >> lgK, j = b & (K - 1);
    xs[l * xst + j] = j < N ? scr[l * N + j] : z0;
  }
  __syncthreads();
  if constexpr (std::is_same<T, double>::value) {
    prefix_segments(xs, xst, lpb, K >> 1);
  } else {
    prefix_warps(xs, xst, lpb, K >> 1);
  }
}

// Orthonormal DST-I of every line in place: xs[l*xst + j] holds x_{j+1}; result y_{k} at
// xs[l*xst + k-1].  FFT route: xst = 2K; the half-length complex FFT works in the line's upper
// half [K, 2K), which holds no data (N < K).  Chirp route: xst = 2K (K the power of two >= n+1),
// scr holds n reals per line.  Dense route: xst = N.
template <typename T>
__device__ void dst_lines(const PassT<T>& P, T* xs, int xst, T* scr) {
  using V = vec2<T>;
  const int N = P.len, lpb = P.lpb;
  const int TH = blockDim.x, tid = threadIdx.x;
  if (P.dim.route == ROUTE_CHIRP) {
    dst_chirp_lines(P, xs, xst, scr);
    return;
  }
  if (P.dim.route == ROUTE_FFT) {
    // DST-I through a real FFT of length K = N+1 (complex FFT of length K2 = K/2):
    //   w_j = sin(pi j/K)(x_j + x_{K-j}) + (x_j - x_{K-j})/2  (x_0 = x_K = 0),  W = DFT_K(w):
    //   y_{2k} = -Im W_k,   y_{2k+1} - y_{2k-1} = Re W_k,  y_1 = Re W_0 / 2.
    // The orthonormal scale h = sqrt(2/K)/2 of the packed outputs is folded into w (sn holds
    // h sin(pi j/K)), so the recombination needs no multiplies.
    const int K = P.dim.K, K2 = K >> 1;
    const T* __restrict__ sn = P.dim.sintab;
    const V* __restrict__ tw2 = P.dim.twK2;
    V* cb = reinterpret_cast<V*>(xs + K);   // line l at cb + l*K (complex)
    const int lk2 = __ffs(K2) - 1;
    const T hh = from_f<T>(0.25f) * P.dim.dsc;   // h / 2 = sqrt(2/K) / 4
    bool input_done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (K2 >= 2) {
        // FP32: the input stage and the twiddle-free first DIT stage in one pass.  The R slots of
        // group g (R = 2 for odd log2 K2, else 4) hold z_m for m = m_lo + r K2/R with g the digit
        // reversal of m_lo; work item m_lo reads its inputs (consecutive lanes, consecutive x),
        // applies the first stage and writes the group as one contiguous run.
        const int R = (lk2 & 1) ? 2 : 4, lgG = lk2 - ((lk2 & 1) ? 1 : 2), G = 1 << lgG;
        for (int b = tid; b < (lpb << lgG); b += TH) {
          const int l = b >> lgG, mlo = b & (G - 1);
          const float* row = xs + l * xst;
          V* x = cb + l * K + R * rev4(mlo, lgG);
          if (R == 2) {
            const V a0 = dst_packed_input(row, mlo, K, sn, hh), a1 = dst_packed_input(row, mlo + G, K, sn, hh);
            x[0] = cadd(a0, a1);
            x[1] = csub(a0, a1);
          } else {
            V a0 = dst_packed_input(row, mlo, K, sn, hh), a1 = dst_packed_input(row, mlo + G, K, sn, hh),
              a2 = dst_packed_input(row, mlo + 2 * G, K, sn, hh), a3 = dst_packed_input(row, mlo + 3 * G, K, sn, hh);
            dit4<false, false>(a0, a1, a2, a3, 0, 1, static_cast<const V*>(nullptr));
            x[0] = a0;
            x[1] = a1;
            x[2] = a2;
            x[3] = a3;
          }
        }
        __syncthreads();
        fft_dit<false>(cb, K, lpb, K2, tw2, false, true);
        input_done = true;
      }
    }
    if (!input_done) {
    for (int b = tid; b < (lpb << lk2); b += TH) {
      const int l = b >> lk2, m = b & (K2 - 1);
      const T* row = xs + l * xst;
      T w[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int j = 2 * m + r;
        T v = from_f<T>(0.0f);
        if (j > 0) {
          const T xj = row[j - 1], xk = row[K - j - 1];
          v = tfma(sn[j], xj + xk, hh * (xj - xk));
        }
        w[r] = v;
      }
      cb[l * K + dif_pos(m, K2)] = mk<V>(w[0], w[1]);
    }
    __syncthreads();
    fft_dit<false>(cb, K, lpb, K2, tw2);
    }
    // recombine pairs (k, K2-k) into W_k, W_{K2-k}; even outputs go to row[2k-1] (odd slots),
    // sc * Re W_k to row[2k] (even slots) for the prefix sum of the odd outputs.
    auto recombine = [&](int l, int k) {
      const int kk = (K2 - k) & (K2 - 1);
      const V* z = cb + l * K;
      const V A = z[k], B = z[kk];
      const V E2 = mk<V>(A.x + B.x, A.y - B.y);
      const V O2 = mk<V>(A.y + B.y, B.x - A.x);
      const V Pw = cmul(ldt(&tw2[K2 + k]), O2);
      T* row = xs + l * xst;
      row[2 * k] = E2.x + Pw.x;                             // sc Re W_k
      if (k > 0) row[2 * k - 1] = -(E2.y + Pw.y);           // y_{2k} = -Im W_k
      if (kk != k) {
        row[2 * kk] = E2.x - Pw.x;                          // sc Re W_{K2-k}
        row[2 * kk - 1] = E2.y - Pw.y;                      // y_{2(K2-k)} = -Im W_{K2-k}
      }
    };
    // slot k in [0, K2/2) of each line: the pair (k, K2-k); slot 0 also takes k = K2/2
    const int H2 = K2 > 1 ? K2 >> 1 : 1, lh2 = __ffs(H2) - 1;
    for (int b = tid; b < (lpb << lh2); b += TH) {
      const int l = b >> lh2, k = b & (H2 - 1);
      recombine(l, k);
      if (k == 0 && K2 > 1) recombine(l, K2 >> 1);
    }
    __syncthreads();
    // prefix sums over the even slots of each line: y_{2k+1} = sum_{i<=k} sc Re W_i - sc Re W_0 / 2.
    // spl threads per line scan contiguous segments; segment offsets by a block-wide shuffle scan.
    if constexpr (std::is_same<T, double>::value) {
      prefix_segments(xs, xst, lpb, K2);
    } else {
      prefix_warps(xs, xst, lpb, K2);
    }
  } else {
    const int K = P.dim.K;
    const T* __restrict__ st = P.dim.sintab;
    const T sc = P.dim.dsc;   // sqrt(2/K), precomputed per dimension
    const T z0 = from_f<T>(0.0f);
    const int tot = lpb * N;
    for (int idx = tid; idx < tot; idx += TH) {
      const int l = idx / N, k = idx - l * N + 1;
      const T* row = xs + l * xst;
      T sacc = z0;
      int ph = k;  // (j * k) mod 2K for j = 1
      for (int j = 1; j <= N; ++j) {
        sacc = tfma(st[ph], row[j - 1], sacc);
        ph += k;
        if (ph >= 2 * K) ph -= 2 * K;
      }
      xs[l * xst + N + k - 1] = sc * sacc;
    }
    dense_copy_back(xs, xst, lpb, N);
  }
}

// ---------------------------------------------------------------------------
// the line-pass kernel
// ---------------------------------------------------------------------------
// Shared memory: ra (lpb*N reals, rounded up to even) then rc (lpb lines of rs reals; rs = 2K on
// the FFT and chirp routes, whose transforms run in place in the padded line (the chirp route
// allocates its rows in pairs), rs = 2N on the dense route: the line, then its outputs).
template <typename T>
__device__ __forceinline__ int rc_stride(const PassT<T>& P) {
  if (P.dim.route == ROUTE_FFT) return 2 * P.dim.K;
  if (P.dim.route == ROUTE_CHIRP) return 2 * P.dim.K;   // K: the power of two >= n + 1
  return 2 * P.len;   // dense: the line, then its outputs (dense_copy_back)
}

// Resident CTAs of 128 threads per SM the register budget allows: 7 for FP64 (72 registers; a
// 1023-line pass fits one wave on 152 SMs), 10 for FP32 (48 registers; its passes are latency
// bound, so more warps help), 6 for the double-float type (85 registers, no spills).
template <typename T> struct PassOcc { static constexpr int ctas = 7; };
template <> struct PassOcc<float> { static constexpr int ctas = 10; };
template <> struct PassOcc<df64> { static constexpr int ctas = 6; };

template <typename T>
__device__ __forceinline__ void pass_run(const PassT<T>& P, VB vb) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = P.len, lpb = P.lpb;
  const int RS = rc_stride(P);
  T* ra = reinterpret_cast<T*>(smraw);
  // an even count of reals before rc keeps every line of rc (and its upper half) aligned for vec2<T>
  T* rc = ra + ((lpb * N + 1) & ~1);
  if (P.g && P.g->done) return;
  if (P.skip && *P.skip) return;
  const TileGeo tg = tile_geo(P, vb.bid);
  const int TH = blockDim.x, tid = threadIdx.x;
  // element loops run over lpb lines of 2^lgnp >= N slots (shift and mask, no division)
  const int lgnp = lg_pad(N), NP = 1 << lgnp, NTP = lpb << lgnp;
  const T* in_a = P.in_a;
  T* out_a = P.out_a;
  if (P.in_sel) in_a = P.in_base + (int64_t)(P.g->j + P.in_sel - 1) * P.vstride;
  if (P.out_sel) out_a = P.out_base + (int64_t)(P.g->j + P.out_sel - 1) * P.vstride;

  if (P.toep_only) {
    tile_load(tg, N, lpb, in_a, rc, RS);
    __syncthreads();
    toeplitz_lines(P, rc, RS);
    tile_store(tg, N, lpb, rc, RS, out_a);
    return;
  }

  if (P.mv) {
    tile_load(tg, N, lpb, in_a, ra, N);
    if (P.first) tile_load(tg, N, lpb, P.e, rc, RS);
    else tile_load(tg, N, lpb, P.in_c, rc, RS);
    __syncthreads();
    const T bd = P.dim.bdiag, bo = P.dim.boff;
    const T seta = from_d<T>(P.seta);
    if (P.first) {
      // ra = x, rc = e  ->  ra = e∘x (kept), rc = x (Toeplitz input), c_out = B x
      for (int idx = tid; idx < NTP; idx += TH) {
        const int l = idx >> lgnp, j = idx & (NP - 1);
        if (j >= N) continue;
        const T x = ra[l * N + j];
        const T e = rc[l * RS + j];
        rc[l * RS + j] = x;
        ra[l * N + j] = e * x;
      }
      __syncthreads();
    }
    // c_out = B c needs c before the Toeplitz product overwrites it; stream it to global.
    if (!P.last) {
      const int tot = tile_total(tg, N, lpb, lgnp);
      for (int idx = tid; idx < tot; idx += TH) {
        int l, j;
        if (!tile_lj(tg, N, lpb, lgnp, idx, l, j)) continue;
        const T v = stencil_B(rc + l * RS, j, N, bd, bo);
        if (l < tg.nvalid) P.out_c[tg.base + l * tg.lstep + (int64_t)j * tg.jstep] = v;
      }
    }
    __syncthreads();
    // rc <- T c in place, then rc <- B a + seta * T c (B a needs ra intact).
    toeplitz_lines(P, rc, RS);
    for (int idx = tid; idx < NTP; idx += TH) {
      const int l = idx >> lgnp, j = idx & (NP - 1);
      if (j >= N) continue;
      const T ba = stencil_B(ra + l * N, j, N, bd, bo);
      rc[l * RS + j] = tfma(seta, rc[l * RS + j], ba);
    }
    __syncthreads();
    if (!P.last) {
      tile_store(tg, N, lpb, rc, RS, out_a);
      return;
    }
    if (P.finish == FIN_ADD_F || P.finish == FIN_RESID) {
      tile_load(tg, N, lpb, P.src, ra, N);
      __syncthreads();
      for (int idx = tid; idx < NTP; idx += TH) {
        const int l = idx >> lgnp, j = idx & (NP - 1);
        if (j >= N) continue;
        T& r = rc[l * RS + j];
        r = (P.finish == FIN_ADD_F) ? r + ra[l * N + j] : ra[l * N + j] - r;
      }
      __syncthreads();
    }
    // fall through to post-processing of rc
  } else {
    tile_load(tg, N, lpb, in_a, rc, RS);
    __syncthreads();
  }

  if (P.post == POST_DST || P.post == POST_DST_MU_DST) {
    dst_lines(P, rc, RS, ra);
    if (P.post == POST_DST_MU_DST) {
      tile_load(tg, N, lpb, P.invmu, ra, N);
      __syncthreads();
      for (int idx = tid; idx < NTP; idx += TH) {
        const int l = idx >> lgnp, j = idx & (NP - 1);
        if (j >= N) continue;
        rc[l * RS + j] *= ra[l * N + j];
      }
      __syncthreads();
      dst_lines(P, rc, RS, ra);
    }
  }
  tile_store(tg, N, lpb, rc, RS, out_a);
}

template <typename T>
struct PassBody {
  using Args = PassT<T>;
  static constexpr int kThreads = PASS_THREADS;
  static constexpr int kCtas = PassOcc<T>::ctas;
  static __device__ __forceinline__ void run(const PassT<T>& P, VB vb) { pass_run<T>(P, vb); }
};
// The wide variant: 256 threads per CTA with the same registers per thread (half the CTAs per SM).
// Lines of a few thousand points per CTA then get twice the threads per transform stage, which
// lifts the warps in flight where the grid has few lines (the FP32 passes at 1023^2 run one or two
// lines per CTA); the autotuner picks it per dimension and element type.
template <typename T>
struct PassBodyW {
  using Args = PassT<T>;
  static constexpr int kThreads = 2 * PASS_THREADS;
  static constexpr int kCtas = PassOcc<T>::ctas / 2;
  static __device__ __forceinline__ void run(const PassT<T>& P, VB vb) { pass_run<T>(P, vb); }
};

template <typename T>
__global__ void __launch_bounds__(PASS_THREADS, PassOcc<T>::ctas) k_pass(const PassT<T> P) {
  pass_run<T>(P, VB{(int)blockIdx.x, (int)gridDim.x});
}

template <typename T>
__global__ void __launch_bounds__(2 * PASS_THREADS, PassOcc<T>::ctas / 2) k_pass_w(const PassT<T> P) {
  pass_run<T>(P, VB{(int)blockIdx.x, (int)gridDim.x});
}

// Hartley passes of the Strang circulant method (POST_HT, POST_HT_D_HT): a kernel of their own, so
// the dense Hartley loop does not weigh on the register allocation of the line-pass kernel.
template <typename T>
__global__ void __launch_bounds__(PASS_THREADS) k_ht_pass(const PassT<T> P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = P.len, lpb = P.lpb;
  const int RS = rc_stride(P);
  T* ra = reinterpret_cast<T*>(smraw);
  T* rc = ra + ((lpb * N + 1) & ~1);
  if (P.g && P.g->done) return;
  const TileGeo tg = tile_geo(P, blockIdx.x);
  const int TH = blockDim.x, tid = threadIdx.x;
  const int lgnp = lg_pad(N), NP = 1 << lgnp, NTP = lpb << lgnp;
  const T* in_a = P.in_a;
  T* out_a = P.out_a;
  if (P.in_sel) in_a = P.in_base + (int64_t)(P.g->j + P.in_sel - 1) * P.vstride;
  if (P.out_sel) out_a = P.out_base + (int64_t)(P.g->j + P.out_sel - 1) * P.vstride;
  tile_load(tg, N, lpb, in_a, rc, RS);
  __syncthreads();
  hartley_lines(P, rc, RS);
  if (P.post == POST_HT_D_HT) {
    tile_load(tg, N, lpb, P.invmu, ra, N);
    __syncthreads();
    for (int idx = tid; idx < NTP; idx += TH) {
      const int l = idx >> lgnp, j = idx & (NP - 1);
      if (j >= N) continue;
      rc[l * RS + j] *= ra[l * N + j];
    }
    __syncthreads();
    hartley_lines(P, rc, RS);
  }
  tile_store(tg, N, lpb, rc, RS, out_a);
}

template <typename T>
size_t pass_smem_bytes(const PassT<T>& p) {
  const size_t ra = ((size_t)p.lpb * p.len + 1) & ~(size_t)1;
  size_t rs = 2 * (size_t)p.len;   // dense: the line and its outputs
  if (p.dim.route == ROUTE_FFT) rs = 2 * (size_t)p.dim.K;
  size_t rows = (size_t)p.lpb;
  if (p.dim.route == ROUTE_CHIRP) {   // rows in pairs: a pair's two rows are its DST buffer
    rs = 2 * (size_t)p.dim.K;
    rows = (rows + 1) & ~(size_t)1;
  }
  return (ra + rows * rs) * sizeof(T);
}

__global__ void k_spectrum(int K, const double* __restrict__ c, double* lam, const double2* __restrict__ twK);
__global__ void k_chirp_spectrum(int M, const double2* __restrict__ b, double2* out, const double2* __restrict__ twM,
                                 double scale);

cudaError_t init_kernel_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pass<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_ht_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pass_w<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pass_w<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pass_w<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_grouped<PassBodyW<double>>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_grouped<PassBodyW<float>>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_grouped<PassBodyW<df64>>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_grouped<PassBody<double>>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_grouped<PassBody<float>>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_grouped<PassBody<df64>>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_chirp_spectrum, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_spectrum, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <typename T>
cudaError_t launch_pass(const PassT<T>& p, cudaStream_t st) {
  const size_t smem = pass_smem_bytes(p);
  const bool wide = p.tpb == 2 * PASS_THREADS;
  if (tl_rec) {
    if (p.post == POST_HT || p.post == POST_HT_D_HT) return cudaErrorNotSupported;   // not grouped
    const unsigned g = p.ntiles > 0 ? (unsigned)p.ntiles : 0u;
    return wide ? record_launch<PassBodyW<T>>(p, g, 2 * PASS_THREADS, smem)
                : record_launch<PassBody<T>>(p, g, PASS_THREADS, smem);
  }
  if (p.ntiles <= 0) return cudaSuccess;
  if (p.post == POST_HT || p.post == POST_HT_D_HT) {
    if constexpr (std::is_same<T, double>::value) {
      k_ht_pass<T><<<(unsigned)p.ntiles, PASS_THREADS, smem, st>>>(p);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;   // the Strang circulant method runs in FP64 only
  }
  if (wide) k_pass_w<T><<<(unsigned)p.ntiles, 2 * PASS_THREADS, smem, st>>>(p);
  else k_pass<T><<<(unsigned)p.ntiles, PASS_THREADS, smem, st>>>(p);
  return cudaGetLastError();
}

template size_t pass_smem_bytes<double>(const PassT<double>&);
template size_t pass_smem_bytes<float>(const PassT<float>&);
template size_t pass_smem_bytes<df64>(const PassT<df64>&);
template cudaError_t launch_pass<double>(const PassT<double>&, cudaStream_t);
template cudaError_t launch_pass<float>(const PassT<float>&, cudaStream_t);
template cudaError_t launch_pass<df64>(const PassT<df64>&, cudaStream_t);

// ---------------------------------------------------------------------------
// setup: circulant spectrum lambda_k = DFT_{2K}(c)_k, k = 0..K (c real symmetric)
// ---------------------------------------------------------------------------
__global__ void k_spectrum(int K, const double* __restrict__ c, double* lam, const double2* __restrict__ twK) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* cb = reinterpret_cast<double2*>(smraw);
  for (int j = threadIdx.x; j < K; j += blockDim.x) cb[j] = make_double2(c[2 * j], c[2 * j + 1]);
  __syncthreads();
  fft_dif(cb, K, 1, K, twK);
  for (int k = threadIdx.x; k <= K / 2; k += blockDim.x) {
    const int kk = (K - k) & (K - 1);
    const double2 A = cb[dif_pos(k, K)], B = cb[dif_pos(kk, K)];
    const double2 E2 = make_double2(A.x + B.x, A.y - B.y);
    const double2 O2 = make_double2(A.y + B.y, B.x - A.x);
    const double2 W = twK[K + k];
    const double2 P = cmul(W, O2);
    lam[k] = 0.5 * (E2.x + P.x);          // Re Y_k
    if (k == 0) lam[K] = 0.5 * (E2.x - P.x);  // Y_K = conj(E2 - W O2)/2 at k = 0
    else if (kk != k) lam[K - k] = 0.5 * (E2.x - P.x);
  }
}

cudaError_t launch_spectrum(int K, const double* c, double* lam, const double2* twK, cudaStream_t st) {
  const size_t smem = (size_t)K * sizeof(double2);
  k_spectrum<<<1, PASS_THREADS, smem, st>>>(K, c, lam, twK);
  return cudaGetLastError();
}

// Stage-packed twiddles on the device (angles reduced exactly in integers first).
__global__ void k_twp(int S, double2* twp) {
  const int n = twp_size(S);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    double num = 0.0, den = 1.0;   // angle = -2 pi num / den
    if (t < S) {
      // find the stage holding t: stage of size s starts at S - s and spans 3 s / 4 entries;
      // entries past the last stage are unused (angle 0)
      int size = S;
      while (size >= 4 && t >= S - size + 3 * (size >> 2)) size >>= 2;
      if (size >= 4) {
        const int q = size >> 2, off = t - (S - size);
        const int r = off / q + 1, i = off - (r - 1) * q;
        num = (double)((r * i) % size);
        den = (double)size;
      }
    } else {
      num = (double)(t - S);
      den = 2.0 * S;
    }
    double sv, cv;
    sincospi(-2.0 * num / den, &sv, &cv);
    twp[t] = make_double2(cv, sv);
  }
}

cudaError_t launch_twp(int S, double2* twp, cudaStream_t st) {
  k_twp<<<(twp_size(S) + 255) / 256, 256, 0, st>>>(S, twp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// setup: spectrum of the chirp kernel of the CHIRP-route DST, left in fft_dif's digit-reversed order
// ---------------------------------------------------------------------------
__global__ void k_chirp_spectrum(int M, const double2* __restrict__ b, double2* out, const double2* __restrict__ twM,
                                 double scale) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* cb = reinterpret_cast<double2*>(smraw);
  for (int j = threadIdx.x; j < M; j += blockDim.x) cb[j] = b[j];
  __syncthreads();
  fft_dif(cb, M, 1, M, twM);
  for (int j = threadIdx.x; j < M; j += blockDim.x) out[j] = make_double2(scale * cb[j].x, scale * cb[j].y);
}

cudaError_t launch_chirp_spectrum(int M, const double2* b, double2* out, const double2* twM, double scale,
                                  cudaStream_t st) {
  k_chirp_spectrum<<<1, PASS_THREADS, (size_t)M * sizeof(double2), st>>>(M, b, out, twM, scale);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fields of step m: e_m = e(G, t_{m+1/2}), Fdt = dt * F^{(m+1/2)}
// ---------------------------------------------------------------------------
__device__ __forceinline__ void unflatten(int64_t idx, int d, const int* n, int* j) {
  for (int i = 0; i < d; ++i) {
    const int64_t q = idx / n[i];
    j[i] = (int)(idx - q * n[i]);
    idx = q;
  }
}

// F = interior restriction of (⊗_l 𝓗_{alpha_l}) f at interior node j, from f on the padded grid
// (Eq. (2.2) applied to the source; Appendix A's 1-D and 2-D forms): the 3^d-point tensor stencil
// with per-dimension weights (alpha/24, 1 - alpha/12, alpha/24), summed one dimension at a time.
__device__ __forceinline__ double fields_hstencil(const FieldDev& F, const double* f, const int* j) {
  const int64_t p0 = F.n[0] + 2, p1 = F.n[1] + 2;
  double acc2 = 0.0;
  for (int o2 = 0; o2 < (F.d > 2 ? 3 : 1); ++o2) {
    double acc1 = 0.0;
    for (int o1 = 0; o1 < (F.d > 1 ? 3 : 1); ++o1) {
      const int64_t i1 = F.d > 1 ? j[1] + o1 : 0, i2 = F.d > 2 ? j[2] + o2 : 0;
      const double* row = f + (i2 * p1 + i1) * p0 + j[0];
      const double v = F.hw[0][0] * (row[0] + row[2]) + F.hw[0][1] * row[1];
      acc1 += (F.d > 1 ? (o1 == 1 ? F.hw[1][1] : F.hw[1][0]) : 1.0) * v;
    }
    acc2 += (F.d > 2 ? (o2 == 1 ? F.hw[2][1] : F.hw[2][0]) : 1.0) * acc1;
  }
  return acc2;
}

// largest number of field terms (e's plus f's) whose per-line coefficients k_fields stages
constexpr int FIELD_RMAX = 32;

struct FieldsArgs {
  FieldDev F;
  const GmresDev* g;
  int64_t m_override;
  double* e_out;
  double* fdt_out;
};

__device__ __forceinline__ void fields_run(const FieldsArgs& A, VB vb) {
  const FieldDev& F = A.F;
  double* e_out = A.e_out;
  double* fdt_out = A.fdt_out;
  const int64_t m = A.m_override >= 0 ? A.m_override : A.g->m;
  if (F.e_dev) {
    const double* em = F.e_dev + m * F.e_step;
    const double* fm = F.f_dev ? F.f_dev + m * F.f_step : nullptr;
    for (int64_t idx = vb.bid * (int64_t)blockDim.x + threadIdx.x; idx < F.n_tot;
         idx += (int64_t)vb.nb * blockDim.x) {
      int j[3] = {0, 0, 0};
      unflatten(idx, F.d, F.n, j);
      if (e_out) e_out[idx] = em[idx];
      if (fdt_out) fdt_out[idx] = fm ? F.dt * fields_hstencil(F, fm, j) : 0.0;
    }
    return;
  }
  const double* etc = F.e_tc + m * F.re;
  const double* ftc = F.f_tc + m * F.rf;
  const int n0 = F.n[0];
  const int64_t nlines = F.n_tot / n0;
  if (F.d > 1 && F.re + F.rf <= FIELD_RMAX && nlines >= 1024 && blockDim.x == 256) {
    // one warp per line along x_1: the line's coefficients c_r prod_{i>=1} phi_{r,i}(x_i) once per
    // line (per lane: a few products), then one FMA per term and element (the FP64 pipe is slow)
    __shared__ double lc[8][FIELD_RMAX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t L = (int64_t)vb.bid * 8 + warp; L < nlines; L += (int64_t)vb.nb * 8) {
      const unsigned q = (unsigned)L;
      const unsigned j1 = F.d > 1 ? q % (unsigned)F.n[1] : 0u, j2 = F.d > 2 ? q / (unsigned)F.n[1] : 0u;
      __syncwarp();
      for (int r = lane; r < F.re + F.rf; r += 32) {
        double p;
        if (r < F.re) {
          p = etc[r] * F.e_sp[1][r * (F.n[1] + 2) + j1 + 1];
          if (F.d > 2) p *= F.e_sp[2][r * (F.n[2] + 2) + j2 + 1];
        } else {
          const int rr = r - F.re;
          p = ftc[rr] * F.f_hsp[1][rr * F.n[1] + j1];
          if (F.d > 2) p *= F.f_hsp[2][rr * F.n[2] + j2];
        }
        lc[warp][r] = p;
      }
      __syncwarp();
      for (int j0 = lane; j0 < n0; j0 += 32) {
        double ev = 0.0, fv = 0.0;
        for (int r = 0; r < F.re; ++r) ev = fma(lc[warp][r], F.e_sp[0][r * (n0 + 2) + j0 + 1], ev);
        for (int r = 0; r < F.rf; ++r) fv = fma(lc[warp][F.re + r], F.f_hsp[0][r * n0 + j0], fv);
        const int64_t idx = L * n0 + j0;
        if (e_out) e_out[idx] = ev;
        if (fdt_out) fdt_out[idx] = F.dt * fv;
      }
    }
    return;
  }
  for (int64_t idx = vb.bid * (int64_t)blockDim.x + threadIdx.x; idx < F.n_tot;
       idx += (int64_t)vb.nb * blockDim.x) {
    int j[3] = {0, 0, 0};
    unflatten(idx, F.d, F.n, j);
    double ev = 0.0;
    for (int r = 0; r < F.re; ++r) {
      double p = etc[r];
      for (int i = 0; i < F.d; ++i) p *= F.e_sp[i][r * (F.n[i] + 2) + j[i] + 1];
      ev += p;
    }
    double fv = 0.0;
    for (int r = 0; r < F.rf; ++r) {
      double p = ftc[r];
      for (int i = 0; i < F.d; ++i) p *= F.f_hsp[i][r * F.n[i] + j[i]];
      fv += p;
    }
    if (e_out) e_out[idx] = ev;
    if (fdt_out) fdt_out[idx] = F.dt * fv;
  }
}

struct FieldsBody {
  using Args = FieldsArgs;
  static constexpr int kThreads = 256, kCtas = 1;
  static __device__ __forceinline__ void run(const FieldsArgs& a, VB vb) { fields_run(a, vb); }
};

__global__ void k_fields(const FieldsArgs A) { fields_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }

cudaError_t launch_fields(const FieldDev& f, const GmresDev* g, int64_t m_override, double* e_out, double* fdt_out,
                          cudaStream_t st) {
  int64_t blocks = (f.n_tot + 255) / 256;
  if (blocks > 4 * 152 * 8) blocks = 4 * 152 * 8;
  const FieldsArgs a{f, g, m_override, e_out, fdt_out};
  if (tl_rec) return record_launch<FieldsBody>(a, (unsigned)blocks, 256, 0);
  k_fields<<<(unsigned)blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

struct PsiArgs {
  int d;
  int n[3];
  int64_t n_tot;
  int rank;
  const double* tc;
  const double* sp[3];
};

__global__ void k_psi(const PsiArgs a, double* out) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.n_tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int j[3] = {0, 0, 0};
    unflatten(idx, a.d, a.n, j);
    double v = 0.0;
    for (int r = 0; r < a.rank; ++r) {
      double p = a.tc[r];
      for (int i = 0; i < a.d; ++i) p *= a.sp[i][r * (a.n[i] + 2) + j[i] + 1];
      v += p;
    }
    out[idx] = v;
  }
}

cudaError_t launch_psi(int d, const int* n, int64_t n_tot, int rank, const double* tc, const double* const* sp,
                       double* out, cudaStream_t st) {
  PsiArgs a;
  a.d = d;
  a.n_tot = n_tot;
  a.rank = rank;
  a.tc = tc;
  for (int i = 0; i < 3; ++i) {
    a.n[i] = i < d ? n[i] : 1;
    a.sp[i] = i < d ? sp[i] : nullptr;
  }
  int64_t blocks = (n_tot + 255) / 256;
  if (blocks > 4 * 152 * 8) blocks = 4 * 152 * 8;
  k_psi<<<(unsigned)blocks, 256, 0, st>>>(a, out);
  return cudaGetLastError();
}

// min / max of e over the interior grid and all half steps (Eq. (dhat)); block partials.
__global__ void k_escan(const FieldDev F, int64_t M, double* partial) {
  __shared__ double smax[256], smin[256];
  double hi = -INFINITY, lo = INFINITY;
  // dense form: every stored value (one slab when e does not depend on t)
  const int64_t total = F.n_tot * (F.e_dev && F.e_step == 0 ? 1 : M);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = t / F.n_tot;
    const int64_t idx = t - m * F.n_tot;
    if (F.e_dev) {
      const double ev = F.e_dev[m * F.e_step + idx];
      hi = fmax(hi, ev);
      lo = fmin(lo, ev);
      continue;
    }
    int j[3] = {0, 0, 0};
    unflatten(idx, F.d, F.n, j);
    const double* etc = F.e_tc + m * F.re;
    double ev = 0.0;
    for (int r = 0; r < F.re; ++r) {
      double p = etc[r];
      for (int i = 0; i < F.d; ++i) p *= F.e_sp[i][r * (F.n[i] + 2) + j[i] + 1];
      ev += p;
    }
    hi = fmax(hi, ev);
    lo = fmin(lo, ev);
  }
  smax[threadIdx.x] = hi;
  smin[threadIdx.x] = lo;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = smax[0];
    partial[2 * blockIdx.x + 1] = smin[0];
  }
}

cudaError_t launch_escan(const FieldDev& f, int64_t M, double* partial, cudaStream_t st) {
  k_escan<<<RED_BLOCKS, 256, 0, st>>>(f, M, partial);
  return cudaGetLastError();
}

struct MuArgs {
  int d;
  int n[3];
  int64_t n_tot;
  double ebar;
  const double* beta[3];
  const double* q[3];
  double eta[3];
};

// 1/mu with mu_J = ebar prod_i beta_i + sum_i eta_i q_i prod_{l!=i} beta_l (Lemma le:eig).
__global__ void k_invmu(const MuArgs a, double* invmu) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.n_tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int j[3] = {0, 0, 0};
    unflatten(idx, a.d, a.n, j);
    double bprod = 1.0;
    for (int i = 0; i < a.d; ++i) bprod *= a.beta[i][j[i]];
    double mu = a.ebar * bprod;
    for (int i = 0; i < a.d; ++i) {
      double p = a.eta[i] * a.q[i][j[i]];
      for (int l = 0; l < a.d; ++l)
        if (l != i) p *= a.beta[l][j[l]];
      mu += p;
    }
    invmu[idx] = 1.0 / mu;
  }
}

cudaError_t launch_invmu(int d, const int* n, int64_t n_tot, double ebar, const double* const* beta,
                         const double* const* q, const double* eta, double* invmu, cudaStream_t st) {
  MuArgs a;
  a.d = d;
  a.n_tot = n_tot;
  a.ebar = ebar;
  for (int i = 0; i < 3; ++i) {
    a.n[i] = i < d ? n[i] : 1;
    a.beta[i] = i < d ? beta[i] : nullptr;
    a.q[i] = i < d ? q[i] : nullptr;
    a.eta[i] = i < d ? eta[i] : 0.0;
  }
  int64_t blocks = (n_tot + 255) / 256;
  if (blocks > 4 * 152 * 8) blocks = 4 * 152 * 8;
  k_invmu<<<(unsigned)blocks, 256, 0, st>>>(a, invmu);
  return cudaGetLastError();
}

// Two-sided preconditioning (Eq. (Pls)): P = ebar I + B^{-1} tau(S) has the eigenvalues mu_k / beta_k
// on the sine basis (beta_k = prod_i beta^{(i)}_{k_i}), so P^{-1/2} = S diag(sqrt(beta/mu)) S and
// P^{-1/2} B^{-1} = S diag(1/sqrt(beta mu)) S.
__global__ void k_tpgm_diag(const MuArgs a, double* pmh, double* pmhb) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.n_tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int j[3] = {0, 0, 0};
    unflatten(idx, a.d, a.n, j);
    double bprod = 1.0;
    for (int i = 0; i < a.d; ++i) bprod *= a.beta[i][j[i]];
    double mu = a.ebar * bprod;
    for (int i = 0; i < a.d; ++i) {
      double p = a.eta[i] * a.q[i][j[i]];
      for (int l = 0; l < a.d; ++l)
        if (l != i) p *= a.beta[l][j[l]];
      mu += p;
    }
    pmh[idx] = sqrt(bprod / mu);
    pmhb[idx] = 1.0 / sqrt(bprod * mu);
  }
}

cudaError_t launch_tpgm_diag(int d, const int* n, int64_t n_tot, double ebar, const double* const* beta,
                             const double* const* q, const double* eta, double* pmh, double* pmhb, cudaStream_t st) {
  MuArgs a;
  a.d = d;
  a.n_tot = n_tot;
  a.ebar = ebar;
  for (int i = 0; i < 3; ++i) {
    a.n[i] = i < d ? n[i] : 1;
    a.beta[i] = i < d ? beta[i] : nullptr;
    a.q[i] = i < d ? q[i] : nullptr;
    a.eta[i] = i < d ? eta[i] : 0.0;
  }
  int64_t blocks = (n_tot + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_tpgm_diag<<<(unsigned)blocks, 256, 0, st>>>(a, pmh, pmhb);
  return cudaGetLastError();
}

// Strang circulant method: pcinv = prod b / (ebar prod b + sum_i eta_i s_i prod_{l!=i} b_l) = 1/p_c
// with b, s the Fourier-basis eigenvalues of s(B_i), s(S_i); binv = 1/prod_i beta^{(i)}.
__global__ void k_spgm_diag(const MuArgs strang, const MuArgs tau_b, double* pcinv, double* binv) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < strang.n_tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int j[3] = {0, 0, 0};
    unflatten(idx, strang.d, strang.n, j);
    double bprod = 1.0, tprod = 1.0;
    for (int i = 0; i < strang.d; ++i) {
      bprod *= strang.beta[i][j[i]];
      tprod *= tau_b.beta[i][j[i]];
    }
    double mu = strang.ebar * bprod;
    for (int i = 0; i < strang.d; ++i) {
      double p = strang.eta[i] * strang.q[i][j[i]];
      for (int l = 0; l < strang.d; ++l)
        if (l != i) p *= strang.beta[l][j[l]];
      mu += p;
    }
    pcinv[idx] = bprod / mu;
    binv[idx] = 1.0 / tprod;
  }
}

cudaError_t launch_spgm_diag(int d, const int* n, int64_t n_tot, double ebar, const double* const* bs,
                             const double* const* ss, const double* eta, const double* const* beta, double* pcinv,
                             double* binv, cudaStream_t st) {
  MuArgs a, t;
  a.d = t.d = d;
  a.n_tot = t.n_tot = n_tot;
  a.ebar = t.ebar = ebar;
  for (int i = 0; i < 3; ++i) {
    a.n[i] = t.n[i] = i < d ? n[i] : 1;
    a.beta[i] = i < d ? bs[i] : nullptr;
    a.q[i] = i < d ? ss[i] : nullptr;
    a.eta[i] = t.eta[i] = i < d ? eta[i] : 0.0;
    t.beta[i] = i < d ? beta[i] : nullptr;
    t.q[i] = nullptr;
  }
  int64_t blocks = (n_tot + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_spgm_diag<<<(unsigned)blocks, 256, 0, st>>>(a, t, pcinv, binv);
  return cudaGetLastError();
}

// u = t (keep = 0) or u += t (keep = 1)
__global__ void k_add_into(double* u, const double* __restrict__ t, int64_t n, int keep) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] = keep ? u[i] + t[i] : t[i];
}

cudaError_t launch_add_into(double* u, const double* t, int64_t n, int keep, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_add_into<<<(unsigned)blocks, 256, 0, st>>>(u, t, n, keep);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// GMRES: classical Gram-Schmidt with one re-orthogonalisation (CGS2), Givens rotations
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;
constexpr int DOT_CHUNK = 4;
// the fused FP32 update-and-dots pass: basis vectors whose values it keeps in registers (more take
// the two-pass form), and elements per thread it handles at a time (measured: 8 x 2 beats 16 x 1,
// which held one element's loads in flight, and 8 x 4, which spills at four CTAs per SM)
constexpr int UPD_KEEP = 8;
constexpr int UPD_U = 2;
// elements per thread whose loads are issued together in the CGS loops (by element size: the
// 8-byte types take two, which keeps the kernels within RED_CTAS CTAs' registers per SM)
template <typename S> struct CgsUnroll { static constexpr int value = sizeof(S) == 4 ? 4 : 2; };
constexpr int RED_CTAS = 4;    // CTAs per SM the CGS kernels are compiled for (RED_BLOCKS = 4 x 152: one wave)

// acc[r] += sum of w[e] V_{i0+r}[e] (r < ni) over this thread's elements e = start, start + stride,
// ... < n.  The loads of CgsUnroll elements are issued before their products, which are added in the
// elements' order (the same sums as one element at a time, with that many times the loads in flight).
template <typename S>
__device__ __forceinline__ void dots_chunk(const S* __restrict__ w, const S* __restrict__ V, int64_t n, int i0,
                                           int ni, int64_t start, int64_t stride, S (&acc)[DOT_CHUNK]) {
  constexpr int CGS_U = CgsUnroll<S>::value;
  for (int64_t idx = start; idx < n; idx += CGS_U * stride) {
    S wv[CGS_U], vv[CGS_U][DOT_CHUNK];
#pragma unroll
    for (int u = 0; u < CGS_U; ++u) {
      const int64_t e = idx + u * stride;
      const bool ok = e < n;
      wv[u] = ok ? w[e] : from_f<S>(0.0f);
#pragma unroll
      for (int r = 0; r < DOT_CHUNK; ++r) vv[u][r] = (ok && r < ni) ? V[(int64_t)(i0 + r) * n + e] : from_f<S>(0.0f);
    }
#pragma unroll
    for (int u = 0; u < CGS_U; ++u)
      if (idx + u * stride < n) {
#pragma unroll
        for (int r = 0; r < DOT_CHUNK; ++r)
          if (r < ni) acc[r] = tfma(wv[u], vv[u][r], acc[r]);
      }
  }
}

// Block sum in FP64 (sh: at least blockDim.x doubles).  Every thread's value goes to shared memory
// and warp 0 adds them, so the FP64 additions (a slow pipe on this part) number ~12 per lane of
// one warp instead of a shuffle tree in every warp.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  __syncthreads();
  sh[threadIdx.x] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    for (int t = threadIdx.x; t < blockDim.x; t += 32) r += sh[t];
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// Last-block completion: every block publishes its partial results, fences, and draws a ticket;
// the block that draws the last one sees all partials and finishes the reduction.  The counter is
// the problem's own (GmresDev.tickets), so concurrent problems never share it; the last block
// resets it for the next launch.
__device__ __forceinline__ bool last_block(unsigned int* tickets, VB vb) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(tickets, 1u);
    s_last = (t == (unsigned)vb.nb - 1u);
    if (s_last) *tickets = 0u;
  }
  __syncthreads();
  return s_last;
}

// h[i] = sum_b partial[i * ld + b], i = 0..jj, by one block (a warp per i); the partials come from
// other SMs, so they are read through L2.
__device__ void reduce_partials(const double* partial, int ld, int jj, double* h, VB vb) {
  const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i <= jj; i += nw) {
    double s = 0.0;
    for (int b = ln; b < vb.nb; b += 32) s += __ldcg(&partial[(int64_t)i * ld + b]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (ln == 0) h[i] = s;
  }
}

// partial[i * ld + blockIdx.x] = sum_{this block's elements} w * V_i, i = 0..j, with w = V_{j+1};
// the last block sums them into h.  Per-element products and per-thread sums in the storage type
// S; block and grid sums in FP64.
template <typename S>
struct DotsArgs {
  const S* V;
  int64_t n;
  GmresDev* g;
  double* partial;
  double* h;
  int ld;
  int pad;
};

template <typename S>
__device__ __forceinline__ void dots_run(const DotsArgs<S>& A, VB vb) {
  const S* __restrict__ V = A.V;
  const int64_t n = A.n;
  GmresDev* g = A.g;
  double* partial = A.partial;
  const int ld = A.ld;
  __shared__ double sh[RED_THREADS];   // block_sum staging (blocks of RED_THREADS threads)
  if (g->done) return;
  const int jj = g->j;
  const S* __restrict__ w = V + (int64_t)(jj + 1) * n;
  for (int i0 = 0; i0 <= jj; i0 += DOT_CHUNK) {
    S acc[DOT_CHUNK];
#pragma unroll
    for (int r = 0; r < DOT_CHUNK; ++r) acc[r] = from_f<S>(0.0f);
    const int ni = min(DOT_CHUNK, jj + 1 - i0);
    dots_chunk<S>(w, V, n, i0, ni, vb.bid * (int64_t)blockDim.x + threadIdx.x, (int64_t)vb.nb * blockDim.x, acc);
#pragma unroll
    for (int r = 0; r < DOT_CHUNK; ++r) {
      if (r < ni) {
        const double s = block_sum(to_d(acc[r]), sh);
        if (threadIdx.x == 0) partial[(int64_t)(i0 + r) * ld + vb.bid] = s;
      }
    }
  }
  if (last_block(&g->tickets, vb)) reduce_partials(partial, ld, jj, A.h, vb);
}

template <typename S>
struct DotsBody {
  using Args = DotsArgs<S>;
  static constexpr int kThreads = RED_THREADS, kCtas = RED_CTAS;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { dots_run<S>(a, vb); }
};

template <typename S>
__global__ void __launch_bounds__(RED_THREADS, RED_CTAS) k_dots(const DotsArgs<S> A) {
  dots_run<S>(A, VB{(int)blockIdx.x, (int)gridDim.x});
}

template <typename S>
cudaError_t launch_dots(const S* V, int64_t n, GmresDev* g, double* partial, int ld, double* h, cudaStream_t st) {
  const DotsArgs<S> a{V, n, g, partial, h, ld, 0};
  if (tl_rec) return record_launch<DotsBody<S>>(a, red_blocks(n), RED_THREADS, 0);
  k_dots<S><<<red_blocks(n), RED_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_dots<double>(const double*, int64_t, GmresDev*, double*, int, double*, cudaStream_t);
template cudaError_t launch_dots<float>(const float*, int64_t, GmresDev*, double*, int, double*, cudaStream_t);
template cudaError_t launch_dots<df64>(const df64*, int64_t, GmresDev*, double*, int, double*, cudaStream_t);

// The Givens step closing Arnoldi column j (one thread): H(:, j) = h1 + h2 with H(j+1, j) = ||w||
// (nsq = ||w||^2), earlier rotations applied, the new rotation, the residual estimate |g_{j+1}|,
// the stop test ||r_j|| <= tol ||r_0|| (or the iteration cap, or breakdown) and the graph condition.
__device__ void givens_column(GmresDev* g, const GivensArgs& a, double nsq) {
  const int j = g->j;
  const double hn = sqrt(nsq);
  double* col = a.H + (int64_t)j * a.ldH;
  for (int i = 0; i <= j; ++i) col[i] = a.h1[i] + a.h2[i];
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double t = a.cs[i] * col[i] + a.sn[i] * col[i + 1];
    col[i + 1] = -a.sn[i] * col[i] + a.cs[i] * col[i + 1];
    col[i] = t;
  }
  const double rr = hypot(col[j], col[j + 1]);
  double c = 1.0, sgv = 0.0;
  if (rr > 0.0) {
    c = col[j] / rr;
    sgv = col[j + 1] / rr;
  }
  a.cs[j] = c;
  a.sn[j] = sgv;
  col[j] = rr;
  col[j + 1] = 0.0;
  a.gv[j + 1] = -sgv * a.gv[j];
  a.gv[j] = c * a.gv[j];
  const double res = fabs(a.gv[j + 1]);
  g->hnorm = hn;
  g->relres = res / g->beta;
  const bool conv = res <= g->tol * g->beta;
  const bool cap = (j + 1) >= g->max_iter;
  const bool brk = !(hn > 0.0);
  if (conv || cap || brk) {
    g->done = 1;
    g->k = j + 1;
    if (!conv && !brk) g->notconv = 1;
    report_cond(a.use_cond, a.gc, false, a.cond, a.cond, false);
  } else {
    g->j = j + 1;
    report_cond(a.use_cond, a.gc, true, a.cond, a.cond, false);
  }
}

// w -= sum_i h_i V_i (w = V_{j+1}); then, with norm_only = false, partial dots of the updated w with
// V_i (CGS2 second pass) finished into h_out by the last block, or, with norm_only = true, ||w||^2
// finished by the last block, which then runs the Givens step.
template <typename S>
struct UpdArgs {
  S* V;
  int64_t n;
  GmresDev* g;
  const double* h;
  double* partial;
  double* h_out;
  int ld;
  int norm_only;
  GivensArgs ga;
};

template <typename S>
__device__ __forceinline__ void update_dots_run(const UpdArgs<S>& A, VB vb) {
  S* V = A.V;
  const int64_t n = A.n;
  GmresDev* g = A.g;
  const double* __restrict__ h = A.h;
  double* partial = A.partial;
  const int ld = A.ld;
  const int norm_only = A.norm_only;
  const GivensArgs& ga = A.ga;
  __shared__ double sh[RED_THREADS];   // block_sum staging (blocks of RED_THREADS threads)
  __shared__ S hs[MAX_ITER_CAP + 1];
  if (g->done) {
    // a finished step (the loop body still runs once after the prologue found r_0 = 0), or, in a
    // grouped launch, a problem that finished before the others: it reports "stop" once
    if (norm_only && vb.bid == 0 && threadIdx.x == 0) report_cond(ga.use_cond, ga.gc, false, ga.cond, ga.cond, false);
    return;
  }
  const int jj = g->j;
  S* w = V + (int64_t)(jj + 1) * n;
  for (int i = threadIdx.x; i <= jj; i += blockDim.x) hs[i] = from_d<S>(h[i]);
  __syncthreads();
  if constexpr (std::is_same<S, float>::value) {
    if (!norm_only && jj < UPD_KEEP) {
      // FP32 basis of at most UPD_KEEP vectors: each element's basis values stay in registers
      // between the update and the second pass's dots, so the basis is read once here instead of
      // twice (same operations in the same order as the two-pass form below); UPD_U elements at a
      // time, their loads issued together
      const int64_t stride = (int64_t)vb.nb * blockDim.x;
      float acc[UPD_KEEP];
#pragma unroll
      for (int i = 0; i < UPD_KEEP; ++i) acc[i] = 0.0f;
      for (int64_t idx = vb.bid * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += UPD_U * stride) {
        float vv[UPD_U][UPD_KEEP], wv[UPD_U];
#pragma unroll
        for (int u = 0; u < UPD_U; ++u) {
          const int64_t e = idx + u * stride;
          const bool ok = e < n;
          wv[u] = ok ? w[e] : 0.0f;
#pragma unroll
          for (int i = 0; i < UPD_KEEP; ++i) vv[u][i] = (ok && i <= jj) ? V[(int64_t)i * n + e] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < UPD_U; ++u)
#pragma unroll
          for (int i = 0; i < UPD_KEEP; ++i)
            if (i <= jj) wv[u] = fmaf(-hs[i], vv[u][i], wv[u]);
#pragma unroll
        for (int u = 0; u < UPD_U; ++u)
          if (idx + u * stride < n) {
            w[idx + u * stride] = wv[u];
#pragma unroll
            for (int i = 0; i < UPD_KEEP; ++i)
              if (i <= jj) acc[i] = fmaf(wv[u], vv[u][i], acc[i]);
          }
      }
#pragma unroll
      for (int i = 0; i < UPD_KEEP; ++i)
        if (i <= jj) {
          const double s = block_sum((double)acc[i], sh);
          if (threadIdx.x == 0) partial[(int64_t)i * ld + vb.bid] = s;
        }
      if (last_block(&g->tickets, vb)) reduce_partials(partial, ld, jj, A.h_out, vb);
      return;
    }
  }
  S nacc = from_f<S>(0.0f);
  {
    // CgsUnroll elements at a time: their loads of each V_i issued together, each element's FMA chain and
    // the norm's sum in the one-element order
    constexpr int CGS_U = CgsUnroll<S>::value;
    const int64_t stride = (int64_t)vb.nb * blockDim.x;
    for (int64_t idx = vb.bid * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += CGS_U * stride) {
      S wv[CGS_U];
#pragma unroll
      for (int u = 0; u < CGS_U; ++u) wv[u] = idx + u * stride < n ? w[idx + u * stride] : from_f<S>(0.0f);
      for (int i = 0; i <= jj; ++i) {
        const S* __restrict__ vi = V + (int64_t)i * n;
        S v[CGS_U];
#pragma unroll
        for (int u = 0; u < CGS_U; ++u) v[u] = idx + u * stride < n ? vi[idx + u * stride] : from_f<S>(0.0f);
#pragma unroll
        for (int u = 0; u < CGS_U; ++u) wv[u] = tfma(-hs[i], v[u], wv[u]);
      }
#pragma unroll
      for (int u = 0; u < CGS_U; ++u)
        if (idx + u * stride < n) {
          w[idx + u * stride] = wv[u];
          nacc = tfma(wv[u], wv[u], nacc);
        }
    }
  }
  if (norm_only) {
    const double s = block_sum(to_d(nacc), sh);
    if (threadIdx.x == 0) partial[vb.bid] = s;
    if (last_block(&g->tickets, vb)) {
      double t = 0.0;
      for (int b = threadIdx.x; b < vb.nb; b += blockDim.x) t += __ldcg(&partial[b]);
      t = block_sum(t, sh);
      if (threadIdx.x == 0) givens_column(g, ga, t);
    }
    return;
  }
  __syncthreads();
  // second Gram-Schmidt pass: dots of the updated w (this block's elements) with V_i
  for (int i0 = 0; i0 <= jj; i0 += DOT_CHUNK) {
    S acc[DOT_CHUNK];
#pragma unroll
    for (int r = 0; r < DOT_CHUNK; ++r) acc[r] = from_f<S>(0.0f);
    const int ni = min(DOT_CHUNK, jj + 1 - i0);
    dots_chunk<S>(w, V, n, i0, ni, vb.bid * (int64_t)blockDim.x + threadIdx.x, (int64_t)vb.nb * blockDim.x, acc);
#pragma unroll
    for (int r = 0; r < DOT_CHUNK; ++r) {
      if (r < ni) {
        const double s = block_sum(to_d(acc[r]), sh);
        if (threadIdx.x == 0) partial[(int64_t)(i0 + r) * ld + vb.bid] = s;
      }
    }
  }
  if (last_block(&g->tickets, vb)) reduce_partials(partial, ld, jj, A.h_out, vb);
}

template <typename S>
struct UpdBody {
  using Args = UpdArgs<S>;
  static constexpr int kThreads = RED_THREADS, kCtas = RED_CTAS;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { update_dots_run<S>(a, vb); }
};

template <typename S>
__global__ void __launch_bounds__(RED_THREADS, RED_CTAS) k_update_dots(const UpdArgs<S> A) {
  update_dots_run<S>(A, VB{(int)blockIdx.x, (int)gridDim.x});
}

template <typename S>
cudaError_t launch_update_dots(S* V, int64_t n, GmresDev* g, const double* h, double* partial, int ld,
                               double* h_out, cudaStream_t st) {
  const UpdArgs<S> a{V, n, g, h, partial, h_out, ld, 0, GivensArgs{}};
  if (tl_rec) return record_launch<UpdBody<S>>(a, red_blocks(n), RED_THREADS, 0);
  k_update_dots<S><<<red_blocks(n), RED_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}
template <typename S>
cudaError_t launch_update_norm_givens(S* V, int64_t n, GmresDev* g, const double* h2, double* partial_norm,
                                      const GivensArgs& ga, cudaStream_t st) {
  const UpdArgs<S> a{V, n, g, h2, partial_norm, nullptr, 0, 1, ga};
  if (tl_rec) return record_launch<UpdBody<S>>(a, red_blocks(n), RED_THREADS, 0);
  k_update_dots<S><<<red_blocks(n), RED_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}
#define TAU_CGS_INST(S)                                                                                          \
  template cudaError_t launch_update_dots<S>(S*, int64_t, GmresDev*, const double*, double*, int, double*,         \
                                             cudaStream_t);                                                       \
  template cudaError_t launch_update_norm_givens<S>(S*, int64_t, GmresDev*, const double*, double*,               \
                                                    const GivensArgs&, cudaStream_t);
TAU_CGS_INST(double)
TAU_CGS_INST(float)
TAU_CGS_INST(df64)
#undef TAU_CGS_INST

// V_{j} <- w / ||w|| where w sits in the slot of V_j (after the Givens step advanced j). When the
// column closed the iteration (done), nothing is scaled.
template <typename S>
struct ScaleNextArgs {
  S* V;
  int64_t n;
  const GmresDev* g;
};

template <typename S>
__device__ __forceinline__ void scale_next_run(const ScaleNextArgs<S>& A, VB vb) {
  const GmresDev* __restrict__ g = A.g;
  if (g->done) return;
  const int j = g->j;
  __shared__ double sinv;   // one FP64 division per block
  if (threadIdx.x == 0) sinv = 1.0 / g->hnorm;
  __syncthreads();
  const S inv = from_d<S>(sinv);
  S* v = A.V + (int64_t)j * A.n;
  constexpr int CGS_U = CgsUnroll<S>::value;
  const int64_t stride = (int64_t)vb.nb * blockDim.x, n = A.n;
  for (int64_t idx = vb.bid * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += CGS_U * stride) {
    S t[CGS_U];
#pragma unroll
    for (int u = 0; u < CGS_U; ++u) t[u] = idx + u * stride < n ? v[idx + u * stride] : from_f<S>(0.0f);
#pragma unroll
    for (int u = 0; u < CGS_U; ++u)
      if (idx + u * stride < n) v[idx + u * stride] = t[u] * inv;
  }
}

template <typename S>
struct ScaleNextBody {
  using Args = ScaleNextArgs<S>;
  static constexpr int kThreads = RED_THREADS, kCtas = RED_CTAS;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { scale_next_run<S>(a, vb); }
};

template <typename S>
__global__ void __launch_bounds__(RED_THREADS, RED_CTAS) k_scale_next(const ScaleNextArgs<S> A) { scale_next_run<S>(A, VB{(int)blockIdx.x, (int)gridDim.x}); }

template <typename S>
cudaError_t launch_scale_next(S* V, int64_t n, const GmresDev* g, cudaStream_t st) {
  const ScaleNextArgs<S> a{V, n, g};
  if (tl_rec) return record_launch<ScaleNextBody<S>>(a, red_blocks(n), RED_THREADS, 0);
  k_scale_next<S><<<red_blocks(n), RED_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_scale_next<double>(double*, int64_t, const GmresDev*, cudaStream_t);
template cudaError_t launch_scale_next<float>(float*, int64_t, const GmresDev*, cudaStream_t);
template cudaError_t launch_scale_next<df64>(df64*, int64_t, const GmresDev*, cudaStream_t);

template <typename S>
struct NormArgs {
  const S* w;
  int64_t n;
  double* partial;
};

template <typename S>
__device__ __forceinline__ void norm_partial_run(const NormArgs<S>& A, VB vb) {
  __shared__ double sh[RED_THREADS];   // block_sum staging (blocks of RED_THREADS threads)
  const S* __restrict__ w = A.w;
  S acc = from_f<S>(0.0f);
  for (int64_t idx = vb.bid * (int64_t)blockDim.x + threadIdx.x; idx < A.n; idx += (int64_t)vb.nb * blockDim.x)
    acc = tfma(w[idx], w[idx], acc);
  const double s = block_sum(to_d(acc), sh);
  if (threadIdx.x == 0) A.partial[vb.bid] = s;
}

template <typename S>
struct NormBody {
  using Args = NormArgs<S>;
  static constexpr int kThreads = RED_THREADS, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { norm_partial_run<S>(a, vb); }
};

template <typename S>
__global__ void __launch_bounds__(RED_THREADS) k_norm_partial(const NormArgs<S> A) {
  norm_partial_run<S>(A, VB{(int)blockIdx.x, (int)gridDim.x});
}

template <typename S>
cudaError_t launch_norm_partial(const S* w, int64_t n, const GmresDev* g, double* partial, cudaStream_t st) {
  (void)g;
  const NormArgs<S> a{w, n, partial};
  if (tl_rec) return record_launch<NormBody<S>>(a, red_blocks(n), RED_THREADS, 0);
  k_norm_partial<S><<<red_blocks(n), RED_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_norm_partial<double>(const double*, int64_t, const GmresDev*, double*, cudaStream_t);
template cudaError_t launch_norm_partial<df64>(const df64*, int64_t, const GmresDev*, double*, cudaStream_t);

// beta = ||r_0||, g_0 = beta, j = 0; done if beta == 0.
__global__ void k_init_beta(GmresDev* g, const double* __restrict__ partial, int nblk, double* gv) {
  __shared__ double sh[RED_THREADS];   // block_sum staging (blocks of RED_THREADS threads)
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    const double beta = sqrt(s);
    g->beta = beta;
    g->j = 0;
    g->k = 0;
    g->relres = 0.0;
    g->hnorm = beta;
    gv[0] = beta;
    g->done = beta > 0.0 ? 0 : 1;
  }
}

template <typename S>
__global__ void k_scale_first(S* V, int64_t n, const GmresDev* __restrict__ g) {
  if (g->done) return;
  __shared__ double sinv;   // one FP64 division per block
  if (threadIdx.x == 0) sinv = 1.0 / g->beta;
  __syncthreads();
  const S inv = from_d<S>(sinv);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x)
    V[idx] *= inv;
}

template <typename S>
cudaError_t launch_init_beta(GmresDev* g, const double* partial, double* gv, S* V, int64_t n, cudaStream_t st) {
  k_init_beta<<<1, 256, 0, st>>>(g, partial, red_blocks(n), gv);   // partials of launch_norm_partial(n)
  k_scale_first<S><<<red_blocks(n), RED_THREADS, 0, st>>>(V, n, g);
  return cudaGetLastError();
}
template cudaError_t launch_init_beta<double>(GmresDev*, const double*, double*, double*, int64_t, cudaStream_t);
template cudaError_t launch_init_beta<df64>(GmresDev*, const double*, double*, df64*, int64_t, cudaStream_t);

// y = R^{-1} g (upper triangular k x k in H after the rotations), then u = x0 + V_k y.
struct BacksolveArgs {
  GmresDev* g;
  const double* H;
  const double* gv;
  double* y;
  int* iters_log;
  int ldH;
  int pad;
};

__device__ __forceinline__ void backsolve_run(const BacksolveArgs& A, VB) {
  if (threadIdx.x != 0) return;
  GmresDev* g = A.g;
  const double* __restrict__ H = A.H;
  const double* __restrict__ gv = A.gv;
  double* y = A.y;
  const int ldH = A.ldH;
  int* iters_log = A.iters_log;
  const int k = g->k;
  for (int i = k - 1; i >= 0; --i) {
    double acc = gv[i];
    for (int c = i + 1; c < k; ++c) acc -= H[(int64_t)c * ldH + i] * y[c];
    y[i] = acc / H[(int64_t)i * ldH + i];
  }
  if (iters_log) iters_log[g->m] = k;
}

struct BacksolveBody {
  using Args = BacksolveArgs;
  static constexpr int kThreads = 32, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { backsolve_run(a, vb); }
};

__global__ void k_backsolve(const BacksolveArgs A) { backsolve_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }

template <typename S>
__global__ void k_update_solution(const GmresDev* __restrict__ g, const double* __restrict__ y,
                                  const S* __restrict__ V, int64_t n, S* u, int x0_prev) {
  __shared__ S ys[MAX_ITER_CAP];
  const int k = g->k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = from_d<S>(y[i]);
  __syncthreads();
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    S v = x0_prev ? u[idx] : from_f<S>(0.0f);
    for (int i = 0; i < k; ++i) v = tfma(ys[i], V[(int64_t)i * n + idx], v);
    u[idx] = v;
  }
}

__global__ void k_advance(GmresDev* g) {
  if (threadIdx.x == 0) g->m += 1;
}

template <typename S>
cudaError_t launch_backsolve_update(GmresDev* g, const double* H, const double* gv, int ldH, double* y, const S* V,
                                    int64_t n, S* u, int x0_prev, int* iters_log, cudaStream_t st) {
  k_backsolve<<<1, 32, 0, st>>>(BacksolveArgs{g, H, gv, y, iters_log, ldH, 0});
  k_update_solution<S><<<red_blocks(n), RED_THREADS, 0, st>>>(g, y, V, n, u, x0_prev);
  k_advance<<<1, 32, 0, st>>>(g);
  return cudaGetLastError();
}
template cudaError_t launch_backsolve_update<double>(GmresDev*, const double*, const double*, int, double*,
                                                     const double*, int64_t, double*, int, int*, cudaStream_t);
template cudaError_t launch_backsolve_update<df64>(GmresDev*, const double*, const double*, int, double*, const df64*,
                                                   int64_t, df64*, int, int*, cudaStream_t);

// Element-wise conversion or copy of whole vectors (setup, per-step fields, API boundary): b = f(a).
template <typename S, typename D>
struct CvtArgs {
  const S* a;   // NULL (copy only): b = 0
  D* b;
  int64_t n;
};

template <typename S, typename D> __device__ __forceinline__ D cvt_elem(S v);
template <> __device__ __forceinline__ df64 cvt_elem<double, df64>(double v) { return from_d<df64>(v); }
template <> __device__ __forceinline__ double cvt_elem<df64, double>(df64 v) { return to_d(v); }
template <> __device__ __forceinline__ float cvt_elem<double, float>(double v) { return (float)v; }
template <> __device__ __forceinline__ double cvt_elem<double, double>(double v) { return v; }

template <typename S, typename D>
__device__ __forceinline__ void cvt_run(const CvtArgs<S, D>& A, VB vb) {
  for (int64_t i = vb.bid * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)vb.nb * blockDim.x)
    A.b[i] = A.a ? cvt_elem<S, D>(A.a[i]) : D{};
}

template <typename S, typename D>
struct CvtBody {
  using Args = CvtArgs<S, D>;
  static constexpr int kThreads = 256, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { cvt_run<S, D>(a, vb); }
};

__global__ void k_d_to_df(const CvtArgs<double, df64> A) { cvt_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }
__global__ void k_df_to_d(const CvtArgs<df64, double> A) { cvt_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }
__global__ void k_f64_to_f32(const CvtArgs<double, float> A) { cvt_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }
__global__ void k_copy(const CvtArgs<double, double> A) { cvt_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }

static unsigned cvt_blocks(int64_t n) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4 * 152 * 8) blocks = 4 * 152 * 8;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

cudaError_t launch_d_to_df(const double* a, df64* b, int64_t n, cudaStream_t st) {
  const CvtArgs<double, df64> c{a, b, n};
  if (tl_rec) return record_launch<CvtBody<double, df64>>(c, cvt_blocks(n), 256, 0);
  k_d_to_df<<<cvt_blocks(n), 256, 0, st>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_df_to_d(const df64* a, double* b, int64_t n, cudaStream_t st) {
  const CvtArgs<df64, double> c{a, b, n};
  if (tl_rec) return record_launch<CvtBody<df64, double>>(c, cvt_blocks(n), 256, 0);
  k_df_to_d<<<cvt_blocks(n), 256, 0, st>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_copy(double* dst, const double* src, int64_t n, cudaStream_t st) {
  const CvtArgs<double, double> c{src, dst, n};
  if (tl_rec) return record_launch<CvtBody<double, double>>(c, cvt_blocks(n), 256, 0);
  k_copy<<<cvt_blocks(n), 256, 0, st>>>(c);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// mixed precision: FP64 iterative refinement around an FP32 flexible GMRES
// ---------------------------------------------------------------------------
cudaError_t launch_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t st) {
  const CvtArgs<double, float> c{a, b, n};
  if (tl_rec) return record_launch<CvtBody<double, float>>(c, cvt_blocks(n), 256, 0);
  k_f64_to_f32<<<cvt_blocks(n), 256, 0, st>>>(c);
  return cudaGetLastError();
}

struct IRArgs {
  IRDev* ir;
  GmresDev* g;          // outer state (ir_finish)
  GmresDev* gin;        // inner FGMRES state (ir_control)
  double* gv_in;
  const double* pnorm;  // ir_control: per-block partial sums of ||r||^2 (nblk of them)
  const double* b;      // first_resid: r = b (bitwise: FP64 or double-float)
  double* r;
  int* iters_log;
  int* sweeps_log;
  GroupCtl* gc;
  int64_t n;
  int nblk;
  int x0_zero;
  int use_cond;
  int pad;
  cudaGraphConditionalHandle cond, cond_in;
};

__device__ __forceinline__ void ir_init_run(const IRArgs& A, VB) {
  IRDev* ir = A.ir;
  if (threadIdx.x == 0) {
    ir->sweep = 0;
    ir->done = 0;
    ir->inner_total = 0;
    ir->skip_resid = 0;
    ir->rho0 = 0.0;
    ir->rho = 0.0;
    ir->rho_prev = 0.0;
    ir->itol_prev = ir->inner_tol;
  }
}

// r = b on the first sweep of a zero initial guess (the residual passes then skip themselves); a
// problem that already converged (a grouped launch runs on while others refine) skips them too.
__device__ __forceinline__ void ir_first_resid_run(const IRArgs& A, VB vb) {
  IRDev* ir = A.ir;
  const bool first = A.x0_zero && ir->sweep == 0 && !ir->done;
  if (first) {
    for (int64_t i = vb.bid * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)vb.nb * blockDim.x)
      A.r[i] = A.b[i];
  }
  if (vb.bid == 0 && threadIdx.x == 0) ir->skip_resid = (first || ir->done) ? 1 : 0;
}

// rho = ||b - A x||; stop when rho <= tol rho_0 or after max_sweeps corrections; otherwise
// start the inner flexible GMRES on v_0 = (b - A x)/rho (beta = 1).
// In the step graph the inner WHILE node lives in the outer loop's body; a handle's default value
// is applied only when the whole graph is launched, so this kernel sets the inner condition for
// every sweep (cond_in) as well as the outer one (cond).
__device__ __forceinline__ void ir_control_run(const IRArgs& A, VB) {
  __shared__ double sh[RED_THREADS];   // block_sum staging (blocks of RED_THREADS threads)
  IRDev* ir = A.ir;
  GmresDev* gin = A.gin;
  if (ir->done) {   // converged earlier: only possible in a grouped launch
    if (threadIdx.x == 0) report_cond(A.use_cond, A.gc, false, A.cond, A.cond_in, true);
    return;
  }
  double s = 0.0;
  for (int b = threadIdx.x; b < A.nblk; b += blockDim.x) s += A.pnorm[b];
  s = block_sum(s, sh);
  if (threadIdx.x != 0) return;
  const double rho = sqrt(s);
  if (ir->sweep == 0) ir->rho0 = rho;
  ir->rho = rho;
  ir->last_rel = ir->rho0 > 0.0 ? rho / ir->rho0 : 0.0;
  const bool conv = !(rho > ir->tol * ir->rho0);
  const bool cap = ir->sweep >= ir->max_sweeps;
  if (conv || cap) {
    ir->done = 1;
    if (!conv) ir->notconv = 1;
    gin->done = 1;
    report_cond(A.use_cond, A.gc, false, A.cond, A.cond_in, true);
    return;
  }
  // Inner target.  The first sweep solves to inner_tol.  A later one asks for the reduction still
  // needed, with a factor 0.3 of margin, need = 0.3 rho0 tol / rho, within [1e-6, 0.5] (an FP32
  // solve cannot resolve much below 1e-6 of its right-hand side).  It never asks for much less than
  // the floor the last sweep ran into: when the last inner solve met its target but the correction
  // reduced the residual by a factor red well above that target (the FP32 operator's own error
  // then limits every sweep), a tighter inner solve costs iterations and buys nothing, so the
  // target is at least red / 2.  (An inner solve stopped by its iteration cap says nothing about
  // that floor.)
  double itol = ir->inner_tol;
  if (ir->sweep > 0) {
    const double need = 0.3 * ir->tol * ir->rho0 / rho;
    const double red = ir->rho_prev > 0.0 ? rho / ir->rho_prev : 0.0;
    const bool met = gin->relres <= 1.0001 * ir->itol_prev;
    const double floor_hit = met && red > 2.0 * ir->itol_prev ? 0.5 * red : 0.0;
    itol = need > floor_hit ? need : floor_hit;
    if (itol < 1e-6) itol = 1e-6;
    if (itol > 0.5) itol = 0.5;
  }
  ir->sweep += 1;
  ir->rho_prev = rho;
  ir->itol_prev = itol;
  gin->tol = itol;
  gin->j = 0;
  gin->k = 0;
  gin->done = 0;
  gin->beta = 1.0;
  gin->hnorm = 1.0;
  A.gv_in[0] = 1.0;
  report_cond(A.use_cond, A.gc, true, A.cond, A.cond_in, true);
}

__device__ __forceinline__ void ir_finish_run(const IRArgs& A, VB) {
  if (threadIdx.x != 0) return;
  const IRDev* ir = A.ir;
  GmresDev* g = A.g;
  if (A.iters_log) A.iters_log[g->m] = ir->inner_total;
  if (A.sweeps_log) A.sweeps_log[g->m] = ir->sweep;
  if (ir->notconv) g->notconv = 1;
  g->relres = ir->last_rel;
  g->m += 1;
}

struct IRInitBody {
  using Args = IRArgs;
  static constexpr int kThreads = 32, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { ir_init_run(a, vb); }
};
struct IRFirstBody {
  using Args = IRArgs;
  static constexpr int kThreads = RED_THREADS, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { ir_first_resid_run(a, vb); }
};
struct IRControlBody {
  using Args = IRArgs;
  static constexpr int kThreads = RED_THREADS, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { ir_control_run(a, vb); }
};
struct IRFinishBody {
  using Args = IRArgs;
  static constexpr int kThreads = 32, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { ir_finish_run(a, vb); }
};

__global__ void k_ir_init(const IRArgs A) { ir_init_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }
__global__ void k_ir_first_resid(const IRArgs A) { ir_first_resid_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }
__global__ void k_ir_control(const IRArgs A) { ir_control_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }
__global__ void k_ir_finish(const IRArgs A) { ir_finish_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }

cudaError_t launch_ir_init(IRDev* ir, cudaStream_t st) {
  IRArgs a{};
  a.ir = ir;
  if (tl_rec) return record_launch<IRInitBody>(a, 1, 32, 0);
  k_ir_init<<<1, 32, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ir_first_resid(IRDev* ir, const double* b, double* r, int64_t n, int x0_zero, cudaStream_t st) {
  IRArgs a{};
  a.ir = ir;
  a.b = b;
  a.r = r;
  a.n = n;
  a.x0_zero = x0_zero;
  if (tl_rec) return record_launch<IRFirstBody>(a, red_blocks(n), RED_THREADS, 0);
  k_ir_first_resid<<<red_blocks(n), RED_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ir_control(IRDev* ir, GmresDev* gin, double* gv_in, const double* pnorm, int64_t n,
                              cudaGraphConditionalHandle cond, cudaGraphConditionalHandle cond_in, int use_cond,
                              GroupCtl* gc, cudaStream_t st) {
  IRArgs a{};
  a.ir = ir;
  a.gin = gin;
  a.gv_in = gv_in;
  a.pnorm = pnorm;
  a.nblk = red_blocks(n);   // partials of launch_norm_partial(n)
  a.cond = cond;
  a.cond_in = cond_in;
  a.use_cond = use_cond;
  a.gc = gc;
  if (tl_rec) return record_launch<IRControlBody>(a, 1, RED_THREADS, 0);
  k_ir_control<<<1, RED_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename S>
struct ScaleF32Args {
  const S* r;
  float* v;
  int64_t n;
  const IRDev* ir;
};

// v = r / rho rounded to FP32 (a double-float r scaled on the FP32 pipes: hi/rho + lo/rho with
// 1/rho as a double-float pair is exact to far below FP32's rounding)
__device__ __forceinline__ float scale_f32(double r, double inv, df64) { return (float)(r * inv); }
__device__ __forceinline__ float scale_f32(df64 r, double, df64 inv) {
  return fmaf(r.hi, inv.hi, fmaf(r.hi, inv.lo, r.lo * inv.hi));
}

template <typename S>
__device__ __forceinline__ void scale_to_f32_run(const ScaleF32Args<S>& A, VB vb) {
  if (A.ir->done) return;
  __shared__ double sinv;   // one FP64 division per block
  if (threadIdx.x == 0) sinv = 1.0 / A.ir->rho;
  __syncthreads();
  const double inv = sinv;
  const df64 inv_df = from_d<df64>(inv);
  for (int64_t i = vb.bid * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)vb.nb * blockDim.x)
    A.v[i] = scale_f32(A.r[i], inv, inv_df);
}

template <typename S>
struct ScaleF32Body {
  using Args = ScaleF32Args<S>;
  static constexpr int kThreads = RED_THREADS, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { scale_to_f32_run<S>(a, vb); }
};

template <typename S>
__global__ void k_scale_to_f32(const ScaleF32Args<S> A) { scale_to_f32_run<S>(A, VB{(int)blockIdx.x, (int)gridDim.x}); }

template <typename S>
cudaError_t launch_scale_to_f32(const S* r, float* v, int64_t n, const IRDev* ir, cudaStream_t st) {
  const ScaleF32Args<S> a{r, v, n, ir};
  if (tl_rec) return record_launch<ScaleF32Body<S>>(a, red_blocks(n), RED_THREADS, 0);
  k_scale_to_f32<S><<<red_blocks(n), RED_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_scale_to_f32<double>(const double*, float*, int64_t, const IRDev*, cudaStream_t);
template cudaError_t launch_scale_to_f32<df64>(const df64*, float*, int64_t, const IRDev*, cudaStream_t);

// x += rho * sum_{i<k} y_i Z_i over the FP32 preconditioned directions Z_i.  The sum runs in
// double-float (about 48 bits, on the FP32 pipes; FP64 conversions and FMAs would run on the slow
// FP64 pipe): the Z_i are exact FP32 vectors, and rounding the correction itself to FP32 would add
// an error of eps_32 |d| whose image under A (not smooth, so A does not cancel on it) is a sizeable
// part of the next residual.  x is FP64 or double-float.
template <typename X> __device__ __forceinline__ void add_to(X& x, df64 d);
template <> __device__ __forceinline__ void add_to<double>(double& x, df64 d) { x += to_d(d); }
template <> __device__ __forceinline__ void add_to<df64>(df64& x, df64 d) { x = x + d; }

// a + b * z with b double-float and z an FP32 value (FMA-exact products of both parts)
__device__ __forceinline__ df64 df_fma_f(df64 b, float z, df64 a) {
  const float p = b.hi * z;
  float e = fmaf(b.hi, z, -p);
  e = fmaf(b.lo, z, e);
  const float h = p + e;
  return a + df64{h, e - (h - p)};
}

template <typename X>
struct UpdXArgs {
  X* x;
  const float* Z;
  const double* y;
  int64_t n;
  const GmresDev* gin;
  IRDev* ir;
};

template <typename X>
__device__ __forceinline__ void update_x_run(const UpdXArgs<X>& A, VB vb) {
  __shared__ df64 ys[MAX_ITER_CAP];
  IRDev* ir = A.ir;
  if (ir->done) return;
  const int k = A.gin->k;
  const double rho = ir->rho;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = from_d<df64>(rho * A.y[i]);
  if (vb.bid == 0 && threadIdx.x == 0) ir->inner_total += k;
  __syncthreads();
  const int64_t n = A.n;
  // four elements at a time: their loads of each Z_i issued together, each element's sum in order
  constexpr int U = 4;
  const int64_t stride = (int64_t)vb.nb * blockDim.x;
  for (int64_t idx = vb.bid * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += U * stride) {
    df64 d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) d[u] = df64{0.0f, 0.0f};
    for (int i = 0; i < k; ++i) {
      const float* __restrict__ zi = A.Z + (int64_t)i * n;
      float z[U];
#pragma unroll
      for (int u = 0; u < U; ++u) z[u] = idx + u * stride < n ? zi[idx + u * stride] : 0.0f;
#pragma unroll
      for (int u = 0; u < U; ++u) d[u] = df_fma_f(ys[i], z[u], d[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (idx + u * stride < n) add_to(A.x[idx + u * stride], d[u]);
  }
}

template <typename X>
struct UpdXBody {
  using Args = UpdXArgs<X>;
  static constexpr int kThreads = RED_THREADS, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { update_x_run<X>(a, vb); }
};

template <typename X>
__global__ void k_update_x(const UpdXArgs<X> A) { update_x_run<X>(A, VB{(int)blockIdx.x, (int)gridDim.x}); }

template <typename X>
cudaError_t launch_update_x(X* x, const float* Z, const double* y, int64_t n, const GmresDev* gin, IRDev* ir,
                            cudaStream_t st) {
  const UpdXArgs<X> a{x, Z, y, n, gin, ir};
  if (tl_rec) return record_launch<UpdXBody<X>>(a, red_blocks(n), RED_THREADS, 0);
  k_update_x<X><<<red_blocks(n), RED_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_update_x<double>(double*, const float*, const double*, int64_t, const GmresDev*, IRDev*,
                                             cudaStream_t);
template cudaError_t launch_update_x<df64>(df64*, const float*, const double*, int64_t, const GmresDev*, IRDev*,
                                           cudaStream_t);

cudaError_t launch_ir_finish(const IRDev* ir, GmresDev* g, int* iters_log, int* sweeps_log, cudaStream_t st) {
  IRArgs a{};
  a.ir = const_cast<IRDev*>(ir);
  a.g = g;
  a.iters_log = iters_log;
  a.sweeps_log = sweeps_log;
  if (tl_rec) return record_launch<IRFinishBody>(a, 1, 32, 0);
  k_ir_finish<<<1, 32, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_backsolve(GmresDev* g, const double* H, const double* gv, int ldH, double* y, cudaStream_t st) {
  const BacksolveArgs a{g, H, gv, y, nullptr, ldH, 0};
  if (tl_rec) return record_launch<BacksolveBody>(a, 1, 32, 0);
  k_backsolve<<<1, 32, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe (bounded loop; 8 independent chains per thread)
// ---------------------------------------------------------------------------
__global__ void k_fp64_peak(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (double)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_fp64_peak(double* out, int blocks, int iters, cudaStream_t st) {
  k_fp64_peak<<<blocks, 256, 0, st>>>(out, iters, 0.999999, 1e-7);
  return cudaGetLastError();
}

}  // namespace tau
