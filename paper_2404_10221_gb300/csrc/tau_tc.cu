// Tensor-core (tcgen05, TF32) DST-I mode product for the FP32 τ solve of the mixed-precision form.
//
// The orthonormal DST-I along one dimension of length n <= 256 is a dense product with the
// symmetric sine matrix S (§3): for every grid line L, y_L[k] = sum_j S[k][j] x_L[j].  With 128
// lines per CTA this is D(128 x N) = X(128 x K) S^T, N = n rounded up to 16, K = n rounded up to 32:
// one tcgen05.mma.kind::tf32 per 8 values of j (M = 128, N columns of fp32 accumulators in tensor
// memory), the operands staged in shared memory in the 8-row x 16-byte core-matrix layout
// (K-major, no swizzle: LBO = 128 B between core matrices along K, SBO = 1 KB between 8-row
// groups), two K-chunks of 32 in flight.  Each chunk's block of S is stored at setup in exactly
// that layout and staged by one bulk asynchronous copy (TMA engine) that completes on the stage's
// mbarrier; the lines go through registers.  Inputs are rounded to TF32 (10-bit mantissa) on the way
// into shared memory, S once at setup, so the product carries a relative error of order 1e-3: the
// flexible GMRES of the mixed form takes the result as its (variable) preconditioner, so this
// changes its iteration count, not the solution it converges to.  The epilogue reads the
// accumulators with tcgen05.ld (warp w owns lanes 32w..32w+31, i.e. lines 32w..32w+31), optionally
// multiplies by a diagonal (the 1/mu of DST·(1/mu)·DST) and stores in place or out of place (each
// CTA reads all of its lines before it writes them).
#include "tau_internal.cuh"

#include <stdint.h>

namespace tau {

constexpr int TC_THREADS = 256;   // two warp groups: each TMEM lane quarter is read by two warps
constexpr int TC_M = 128;        // lines per CTA (accumulator rows = TMEM lanes)
constexpr int TC_KC = 32;        // K values per shared-memory stage (four MMAs of K = 8)
constexpr int TC_WAIT = 4000000; // polls of an mbarrier before the kernel gives up

struct TcArgs {
  int n, ax, inner, N, Kp, nalloc;
  int64_t nlines;
  const float* S;        // per K-chunk c: the N x 32 block of S in the shared-memory core-matrix
                         // layout (N*32 floats at c*N*32), TF32-rounded, zero padded
  const float* in;
  float* in_base;
  int in_sel;
  float* out;
  float* out_base;
  int out_sel;
  int64_t vstride;
  const GmresDev* g;
  const int* skip;
  const float* mul;      // non-null: multiply the result by mul (same layout as the vector)
  int* err;              // set to 1 when an mbarrier wait gives up
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, k) in a K-major no-swizzle tile of 32 fp32 per row
__device__ __forceinline__ int cm_off(int row, int k) {
  return (row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor: start address, LBO, SBO (bytes, multiples of 16), descriptor
// version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ float to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, int limit = TC_WAIT) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(32);
  }
  return false;
}

// Bulk asynchronous copy (TMA engine, untiled) of `bytes` from global to shared memory, completing
// on the mbarrier `bar`; both addresses 16-byte aligned, bytes a multiple of 16.  The caller has
// announced the bytes on the barrier with expect_tx.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bars_init(uint64_t* bars, int count) {
  for (int i = 0; i < count; ++i)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[i])), "r"(1));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

template <bool MUL>
__global__ void __launch_bounds__(TC_THREADS) k_tc_mode(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  if ((a.g && a.g->done) || (a.skip && *a.skip)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N, n = a.n;
  // dimension 0 (lines contiguous): D[k][line] = S X^T (A = S, M = 128 k per tile, B = the lines,
  // N = 128), so TMEM lanes run along k and the stores along each line coalesce; other dimensions
  // (lines interleaved): D[line][k] = X S^T (A = the lines, B = S), lanes run across lines
  const bool flip = a.ax == 0;
  const int MT = flip ? N >> 7 : 1;
  const int stage = TC_M * TC_KC * 4 + N * TC_KC * 4;   // line tile, then the S tile
  // bars[0..1]: MMAs of the stage done; bars[2..3]: the stage's S block landed
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * stage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * stage + 32);
  const int64_t L0 = (int64_t)blockIdx.x * TC_M;
  const float* x = a.in_sel ? a.in_base + (int64_t)(a.g->j + a.in_sel - 1) * a.vstride : a.in;
  float* y = a.out_sel ? a.out_base + (int64_t)(a.g->j + a.out_sel - 1) * a.vstride : a.out;
  // other dimensions: thread tid owns line L0 + (tid mod 128) (element j at base + j*jstep) and
  // stages half of its values of each chunk; warp w reads TMEM lanes 32 (w mod 4).. and every other
  // block of 16 accumulator columns (hf = w / 4)
  const int ln = tid & (TC_M - 1), hf = tid >> 7;
  const int64_t L = L0 + ln;
  const bool live = L < a.nlines;
  int64_t base = 0, jstep = 1;
  if (live && !flip) {
    const int64_t sl = L / a.inner, b = L - sl * a.inner;
    base = sl * n * a.inner + b;
    jstep = a.inner;
  }
  if (tid == 0) bars_init(bars, 4);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.nalloc));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  // kind::tf32: D f32 (bits 4-5 = 1), A and B tf32 (bits 7-9, 10-12 = 2), both K-major,
  // N >> 3 at bit 17, M >> 4 at bit 24
  const int nmma = flip ? TC_M : N;
  const uint32_t idesc =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nmma >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
  const int C = a.Kp / TC_KC;
  // the 16 line values this thread stages per chunk, loaded one chunk ahead (software pipeline:
  // chunk c+1's loads are in flight during chunk c's copy of S, barrier and MMA issue)
  //   dimension 0: warp w stages lines 16w..16w+15, one load instruction covering 8 lines x 4
  //   consecutive j (8 sectors) whose shared-memory stores hit 32 distinct banks;
  //   other dimensions: half of this thread's line, stored as four 16-byte core-matrix rows
  float nv[16];
  auto load_chunk = [&](int c) {
    const int j0 = c * TC_KC;
    if (flip) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int row = 16 * warp + 8 * (i & 1) + (lane >> 2), k = 4 * (i >> 1) + (lane & 3), j = j0 + k;
        const int64_t Lr = L0 + row;
        nv[i] = (Lr < a.nlines && j < n) ? x[Lr * n + j] : 0.0f;
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int j = j0 + 16 * hf + jj;
        nv[jj] = (live && j < n) ? x[base + (int64_t)j * jstep] : 0.0f;
      }
    }
  };
  load_chunk(0);
  bool ok = true;
  int pend = -1;   // chunk whose S copy is in flight and not yet seen complete
  int lastc = -1;  // last chunk whose MMAs were committed
  for (int c = 0; c < C; ++c) {
    const int s = c & 1;
    unsigned char* sx = sm + s * stage;          // 128 lines x 32
    unsigned char* ss = sx + TC_M * TC_KC * 4;   // N rows of S x 32
    // the MMAs of chunk c - 2 read this stage: wait for their commit (the outcome is made uniform
    // over the block, so every thread takes the same barriers)
    if (c >= 2) {
      ok = __syncthreads_and(bar_wait(smem_u32(&bars[s]), ((c - 2) >> 1) & 1) ? 1 : 0) != 0;
      if (!ok) break;
    }
    // the chunk's block of S is stored in the shared-memory layout: one bulk copy (N*128 bytes from
    // a 16-byte aligned offset into a 1 KB aligned stage), in flight while the lines are staged
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)(N * TC_KC * 4);
      bar_expect_tx(smem_u32(&bars[2 + s]), bytes);
      bulk_g2s(smem_u32(ss), a.S + (int64_t)c * N * TC_KC, bytes, smem_u32(&bars[2 + s]));
    }
    pend = c;
    if (flip) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int row = 16 * warp + 8 * (i & 1) + (lane >> 2), k = 4 * (i >> 1) + (lane & 3);
        *reinterpret_cast<float*>(sx + cm_off(row, k)) = to_tf32(nv[i]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 w = make_float4(to_tf32(nv[4 * q]), to_tf32(nv[4 * q + 1]), to_tf32(nv[4 * q + 2]),
                                     to_tf32(nv[4 * q + 3]));
        *reinterpret_cast<float4*>(sx + cm_off(ln, 16 * hf + 4 * q)) = w;
      }
    }
    if (c + 1 < C) load_chunk(c + 1);
    // the lines' stores made visible to the tensor cores, and the S block landed
    asm volatile("fence.proxy.async.shared::cta;");
    ok = __syncthreads_and(bar_wait(smem_u32(&bars[2 + s]), (c >> 1) & 1) ? 1 : 0) != 0;
    if (!ok) break;
    pend = -1;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int q = 0; q < TC_KC / 8; ++q) {
        const uint32_t acc = (c > 0 || q > 0) ? 1u : 0u;
        for (int t = 0; t < MT; ++t) {
          // A: 128 rows (lines, or S rows 128t..) at K step q; B: N (or 128) rows
          const uint64_t da = flip ? smem_desc(smem_u32(ss) + t * 16384 + 256 * q, 128, 1024)
                                   : smem_desc(smem_u32(sx) + 256 * q, 128, 1024);
          const uint64_t db = flip ? smem_desc(smem_u32(sx) + 256 * q, 128, 1024)
                                   : smem_desc(smem_u32(ss) + 256 * q, 128, 1024);
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + 128u * t),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&bars[s])));
    }
    lastc = c;
  }
  // the last commit tracks every MMA of the CTA
  if (ok) ok = __syncthreads_and(bar_wait(smem_u32(&bars[lastc & 1]), (lastc >> 1) & 1) ? 1 : 0) != 0;
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 1);
    // give the copy and the MMAs in flight a further bounded wait before the shared memory and the
    // accumulators are released
    if (pend >= 0) bar_wait(smem_u32(&bars[2 + (pend & 1)]), (pend >> 1) & 1);
    if (lastc >= 0) bar_wait(smem_u32(&bars[lastc & 1]), (lastc >> 1) & 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const float* __restrict__ mul = a.mul;
    for (int t = 0; t < MT; ++t) {
      const int ncol = flip ? TC_M : N;
      for (int cc = 16 * hf; cc < ncol; cc += 32) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(128 * t + cc);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float r[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = __uint_as_float(v[q]);
        if (flip) {   // lane = k, columns = lines
          const int k = 128 * t + 32 * (warp & 3) + lane;
          if (k < n) {
            if (MUL) {   // the diagonal first (independent loads), then the stores
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const int64_t Lq = L0 + cc + q;
                r[q] *= Lq < a.nlines ? __ldg(&mul[Lq * n + k]) : 0.0f;
              }
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int64_t Lq = L0 + cc + q;
              if (Lq < a.nlines) y[Lq * n + k] = r[q];
            }
          }
        } else if (live) {   // lane = line, columns = k
          if (MUL) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int k = cc + q;
              r[q] *= k < n ? __ldg(&mul[base + (int64_t)k * jstep]) : 0.0f;
            }
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int k = cc + q;
            if (k < n) y[base + (int64_t)k * jstep] = r[q];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.nalloc));
}

// ---------------------------------------------------------------------------
// Split-TF32 Toeplitz matvec pass of the FP32 inner solve (all dimensions n <= 256)
// ---------------------------------------------------------------------------
// One pass of the matvec chain along dimension ax, as in the line-pass kernel: with the channels
// a (first pass: e∘x) and c (first pass: x),
//     a' = B_ax a + seta T_ax c,      c' = B_ax c   (not on the last pass; the last stores a'),
// B_ax the tridiagonal stencil (bd, bo) along the line and T_ax the Toeplitz matrix of the FCD
// weights.  T c is a dense product on the tensor cores with FP32-level accuracy from split TF32
// operands: c = c_hi + c_lo, T = T_hi + T_lo (each part TF32), T c ~ T_hi c_hi + T_hi c_lo + T_lo c_hi
// (the dropped T_lo c_lo is ~2^-22 relative).  K-chunks of 16 (two MMA K-steps, three products
// each), core-matrix layout with 512-byte row groups; the chunk's T_hi and T_lo blocks arrive by
// two bulk asynchronous copies on the stage's mbarrier.  The stencil reads a and c (neighbours
// included) from global memory in the epilogue, so the pass writes new channel buffers.
constexpr int TM_KC = 16;

struct TcMvArgs {
  int n, ax, inner, N, Kp, nalloc;
  int64_t nlines;
  const float* Thi;      // per K-chunk of 16: N x 16 block of T_hi in the core-matrix layout
  const float* Tlo;
  const float* c_in;     // Toeplitz input (first pass: x)
  float* c_base;
  int c_sel;
  const float* a_in;     // not first: channel a
  const float* e;        // first pass: e
  float* out_a;          // last: the result; else channel a'
  float* out_base;
  int out_sel;
  float* out_c;          // not last: channel c'
  int first, last;
  float bd, bo, seta;
  int64_t vstride;
  const GmresDev* g;
  const int* skip;
  int* err;
};

__device__ __forceinline__ int cm16(int row, int k) {
  return (row >> 3) * 512 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
  hi = to_tf32(v);
  lo = to_tf32(v - hi);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__global__ void __launch_bounds__(TC_THREADS) k_tc_mv(const TcMvArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  if ((a.g && a.g->done) || (a.skip && *a.skip)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N, n = a.n;
  const bool flip = a.ax == 0;
  const int MT = flip ? N >> 7 : 1;
  const int xt = TC_M * TM_KC * 4, tt = N * TM_KC * 4;   // line tile, T tile (bytes)
  const int stage = 2 * xt + 2 * tt;                     // x_hi, x_lo, T_hi, T_lo
  // bars[0..1]: MMAs of the stage done; bars[2..3]: the stage's T_hi, T_lo blocks landed
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * stage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * stage + 32);
  const int64_t L0 = (int64_t)blockIdx.x * TC_M;
  const float* cin = a.c_sel ? a.c_base + (int64_t)(a.g->j + a.c_sel - 1) * a.vstride : a.c_in;
  float* outa = a.out_sel ? a.out_base + (int64_t)(a.g->j + a.out_sel - 1) * a.vstride : a.out_a;
  const int ln = tid & (TC_M - 1), hf = tid >> 7;
  const int64_t L = L0 + ln;
  const bool live = L < a.nlines;
  int64_t base = 0, jstep = 1;
  if (live && !flip) {
    const int64_t sl = L / a.inner, b = L - sl * a.inner;
    base = sl * n * a.inner + b;
    jstep = a.inner;
  }
  if (tid == 0) bars_init(bars, 4);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.nalloc));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const int nmma = flip ? TC_M : N;
  const uint32_t idesc =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nmma >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
  const int C = a.Kp / TM_KC;
  // the 8 values this thread stages per chunk, loaded one chunk ahead (dimension 0: warp w stages
  // lines 16w..16w+15, 8 lines x 4 consecutive j per instruction; other dimensions: half of this
  // thread's line as two 16-byte core-matrix rows, hi and lo)
  float nv[8];
  auto load_chunk = [&](int c) {
    const int j0 = c * TM_KC;
    if (flip) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = 16 * warp + 8 * (i & 1) + (lane >> 2), k = 4 * (i >> 1) + (lane & 3), j = j0 + k;
        const int64_t Lr = L0 + row;
        nv[i] = (Lr < a.nlines && j < n) ? cin[Lr * n + j] : 0.0f;
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int j = j0 + 8 * hf + jj;
        nv[jj] = (live && j < n) ? cin[base + (int64_t)j * jstep] : 0.0f;
      }
    }
  };
  load_chunk(0);
  bool ok = true;
  int pend = -1;   // chunk whose T copies are in flight and not yet seen complete
  int lastc = -1;  // last chunk whose MMAs were committed
  for (int c = 0; c < C; ++c) {
    const int s = c & 1;
    unsigned char* sxh = sm + s * stage;
    unsigned char* sxl = sxh + xt;
    unsigned char* sth = sxl + xt;
    unsigned char* stl = sth + tt;
    if (c >= 2) {
      ok = __syncthreads_and(bar_wait(smem_u32(&bars[s]), ((c - 2) >> 1) & 1) ? 1 : 0) != 0;
      if (!ok) break;
    }
    // the chunk's T_hi and T_lo blocks (N*64 bytes each, 16-byte aligned offsets, stored in the
    // shared-memory layout): two bulk copies on one barrier, in flight while the lines are staged
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)tt;
      bar_expect_tx(smem_u32(&bars[2 + s]), 2 * bytes);
      bulk_g2s(smem_u32(sth), a.Thi + (int64_t)c * N * TM_KC, bytes, smem_u32(&bars[2 + s]));
      bulk_g2s(smem_u32(stl), a.Tlo + (int64_t)c * N * TM_KC, bytes, smem_u32(&bars[2 + s]));
    }
    pend = c;
    if (flip) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = 16 * warp + 8 * (i & 1) + (lane >> 2), k = 4 * (i >> 1) + (lane & 3);
        float hi, lo;
        split_tf32(nv[i], hi, lo);
        *reinterpret_cast<float*>(sxh + cm16(row, k)) = hi;
        *reinterpret_cast<float*>(sxl + cm16(row, k)) = lo;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float h[4], l[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) split_tf32(nv[4 * q + r], h[r], l[r]);
        *reinterpret_cast<float4*>(sxh + cm16(ln, 8 * hf + 4 * q)) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(sxl + cm16(ln, 8 * hf + 4 * q)) = make_float4(l[0], l[1], l[2], l[3]);
      }
    }
    if (c + 1 < C) load_chunk(c + 1);
    asm volatile("fence.proxy.async.shared::cta;");
    ok = __syncthreads_and(bar_wait(smem_u32(&bars[2 + s]), (c >> 1) & 1) ? 1 : 0) != 0;
    if (!ok) break;
    pend = -1;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int q = 0; q < TM_KC / 8; ++q) {
        for (int t = 0; t < MT; ++t) {
          const uint32_t d = tmem + 128u * t;
          const uint32_t xo = 256 * q, to = t * 8192 + 256 * q;
          // T c ~ T_hi c_hi + T_hi c_lo + T_lo c_hi
          const uint64_t xh = smem_desc(smem_u32(sxh) + xo, 128, 512), xl = smem_desc(smem_u32(sxl) + xo, 128, 512);
          const uint64_t th = smem_desc(smem_u32(sth) + (flip ? to : xo), 128, 512);
          const uint64_t tl = smem_desc(smem_u32(stl) + (flip ? to : xo), 128, 512);
          const uint32_t acc0 = (c > 0 || q > 0) ? 1u : 0u;
          if (flip) {
            mma_tf32(d, th, xh, idesc, acc0);
            mma_tf32(d, th, xl, idesc, 1u);
            mma_tf32(d, tl, xh, idesc, 1u);
          } else {
            mma_tf32(d, xh, th, idesc, acc0);
            mma_tf32(d, xl, th, idesc, 1u);
            mma_tf32(d, xh, tl, idesc, 1u);
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&bars[s])));
    }
    lastc = c;
  }
  if (ok) ok = __syncthreads_and(bar_wait(smem_u32(&bars[lastc & 1]), (lastc >> 1) & 1) ? 1 : 0) != 0;
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 1);
    if (pend >= 0) bar_wait(smem_u32(&bars[2 + (pend & 1)]), (pend >> 1) & 1);
    if (lastc >= 0) bar_wait(smem_u32(&bars[lastc & 1]), (lastc >> 1) & 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const float* __restrict__ av = a.first ? nullptr : a.a_in;
    const float* __restrict__ ev = a.e;
    const float bd = a.bd, bo = a.bo, seta = a.seta;
    const bool fst = a.first != 0, lst = a.last != 0;
    // the channels at index o (a = e∘x on the first pass, c = x there)
    auto ach = [&](int64_t o) -> float { return fst ? __ldg(&ev[o]) * cin[o] : __ldg(&av[o]); };
    for (int t = 0; t < MT; ++t) {
      const int ncol = flip ? TC_M : N;
      for (int cc = 16 * hf; cc < ncol; cc += 32) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(128 * t + cc);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (flip) {
          // lane = k along the 16 lines L0 + cc + q: each lane loads its own a_k, c_k of all 16 lines
          // before any use; the neighbours come from the adjacent lanes, and the two beyond the
          // warp's 32 columns (k-1 for lane 0, k+1 for lane 31) from one halo load per channel, lane q
          // holding line q's left value and lane 16 + q its right one
          const int kb = 128 * t + 32 * (warp & 3), k = kb + lane;
          const int hk = lane < 16 ? kb - 1 : kb + 32;
          const int64_t Lh = L0 + cc + (lane & 15);
          const bool vh = Lh < a.nlines && hk >= 0 && hk < n;
          const float ha = vh ? ach(Lh * n + hk) : 0.0f;
          const float hc = (!lst && vh) ? cin[Lh * n + hk] : 0.0f;
          float ak[16], ck[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int64_t Lq = L0 + cc + q;
            const bool valid = Lq < a.nlines && k < n;
            const int64_t o = Lq * n + k;
            ak[q] = valid ? ach(o) : 0.0f;
            ck[q] = (!lst && valid) ? cin[o] : 0.0f;
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int64_t Lq = L0 + cc + q;
            const bool valid = Lq < a.nlines && k < n;
            const int64_t o = Lq * n + k;
            float al = __shfl_up_sync(0xffffffffu, ak[q], 1), ar = __shfl_down_sync(0xffffffffu, ak[q], 1);
            float cl = __shfl_up_sync(0xffffffffu, ck[q], 1), cr = __shfl_down_sync(0xffffffffu, ck[q], 1);
            const int src = lane == 0 ? q : 16 + q;
            const float hav = __shfl_sync(0xffffffffu, ha, src), hcv = __shfl_sync(0xffffffffu, hc, src);
            if (lane == 0) {
              al = hav;
              cl = hcv;
            }
            if (lane == 31) {
              ar = hav;
              cr = hcv;
            }
            if (valid) {
              const float res = fmaf(seta, __uint_as_float(v[q]), fmaf(bd, ak[q], bo * (al + ar)));
              if (lst) {
                outa[o] = res;
              } else {
                a.out_a[o] = res;
                a.out_c[o] = fmaf(bd, ck[q], bo * (cl + cr));
              }
            }
          }
        } else if (live) {
          // lane = line, columns k = cc..cc+15: the channels' runs k = cc-1..cc+16 are loaded once
          float ar[18], cr[18];
#pragma unroll
          for (int r = 0; r < 18; ++r) {
            const int k = cc - 1 + r;
            const bool in = k >= 0 && k < n;
            const int64_t o = base + (int64_t)k * jstep;
            ar[r] = in ? ach(o) : 0.0f;
            cr[r] = (!lst && in) ? cin[o] : 0.0f;
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int k = cc + q;
            if (k >= n) continue;
            const int64_t o = base + (int64_t)k * jstep;
            const float res = fmaf(seta, __uint_as_float(v[q]), fmaf(bd, ar[q + 1], bo * (ar[q] + ar[q + 2])));
            if (lst) {
              outa[o] = res;
            } else {
              a.out_a[o] = res;
              a.out_c[o] = fmaf(bd, cr[q + 1], bo * (cr[q] + cr[q + 2]));
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.nalloc));
}

size_t tm_smem_bytes(int N) { return 2 * (size_t)(2 * TC_M * TM_KC * 4 + 2 * N * TM_KC * 4) + 64; }

cudaError_t launch_tc_mv(const PassT<float>& p, const TcTab& t, const float* c_in, float* c_base, int c_sel,
                         const float* a_in, float* out_a, float* out_base, int out_sel, float* out_c, bool first,
                         bool last, cudaStream_t st) {
  TcMvArgs a{};
  a.n = t.n;
  a.ax = p.ax;
  a.inner = (int)p.inner;
  a.N = t.N;
  a.Kp = t.Kp16;
  a.nalloc = t.nalloc;
  a.nlines = p.nlines;
  a.Thi = t.Thi;
  a.Tlo = t.Tlo;
  a.c_in = c_in;
  a.c_base = c_base;
  a.c_sel = c_sel;
  a.a_in = a_in;
  a.e = p.e;
  a.out_a = out_a;
  a.out_base = out_base;
  a.out_sel = out_sel;
  a.out_c = out_c;
  a.first = first;
  a.last = last;
  a.bd = p.dim.bdiag;
  a.bo = p.dim.boff;
  a.seta = (float)p.seta;
  a.vstride = p.vstride;
  a.g = p.g;
  a.skip = p.skip;
  a.err = t.err;
  const unsigned grid = (unsigned)((p.nlines + TC_M - 1) / TC_M);
  k_tc_mv<<<grid, TC_THREADS, tm_smem_bytes(t.N), st>>>(a);
  return cudaGetLastError();
}

// Self-test of the bounded wait: one CTA waits on an mbarrier that nothing arrives at; the wait must
// give up after `polls` polls and report it (no fault, no hang).
__global__ void k_wait_selftest(int polls, int* gave_up) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
  __syncthreads();
  const bool ok = __syncthreads_and(bar_wait(smem_u32(&bar), 0, polls) ? 1 : 0) != 0;
  if (threadIdx.x == 0) *gave_up = ok ? 0 : 1;
}

cudaError_t launch_wait_selftest(int polls, int* gave_up, cudaStream_t st) {
  k_wait_selftest<<<1, 64, 0, st>>>(polls, gave_up);
  return cudaGetLastError();
}

size_t tc_smem_bytes(int N) { return 2 * (size_t)(TC_M * TC_KC * 4 + N * TC_KC * 4) + 64; }

cudaError_t init_tc_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_mode<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes(256));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tc_mode<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes(256));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_mv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tm_smem_bytes(256));
}

cudaError_t launch_tc_dst(const PassT<float>& p, const TcTab& t, const float* mul, bool from_out, cudaStream_t st) {
  TcArgs a{};
  a.n = t.n;
  a.ax = p.ax;
  a.inner = (int)p.inner;
  a.N = t.N;
  a.Kp = t.Kp;
  a.nalloc = t.nalloc;
  a.nlines = p.nlines;
  a.S = t.S;
  if (from_out) {   // second product of DST·(1/mu)·DST: in place on the output
    a.in = p.out_a;
    a.in_base = p.out_base;
    a.in_sel = p.out_sel;
  } else {
    a.in = p.in_a;
    a.in_base = p.in_base;
    a.in_sel = p.in_sel;
  }
  a.out = p.out_a;
  a.out_base = p.out_base;
  a.out_sel = p.out_sel;
  a.vstride = p.vstride;
  a.g = p.g;
  a.skip = p.skip;
  a.mul = mul;
  a.err = t.err;
  const unsigned grid = (unsigned)((p.nlines + TC_M - 1) / TC_M);
  if (mul)
    k_tc_mode<true><<<grid, TC_THREADS, tc_smem_bytes(t.N), st>>>(a);
  else
    k_tc_mode<false><<<grid, TC_THREADS, tc_smem_bytes(t.N), st>>>(a);
  return cudaGetLastError();
}

}  // namespace tau
