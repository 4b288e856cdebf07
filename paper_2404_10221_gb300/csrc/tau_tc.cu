// Tensor-core (tcgen05, TF32) DST-I mode product for the FP32 τ solve of the mixed-precision form.
//
// The orthonormal DST-I along one dimension of length n <= 256 is a dense product with the
// symmetric sine matrix S (§3): for every grid line L, y_L[k] = sum_j S[k][j] x_L[j].  With 128
// lines per CTA this is D(128 x N) = X(128 x K) S^T, N = n rounded up to 16, K = n rounded up to 32:
// one tcgen05.mma.kind::tf32 per 8 values of j (M = 128, N columns of fp32 accumulators in tensor
// memory), the operands staged in shared memory in the 8-row x 16-byte core-matrix layout
// (K-major, no swizzle: LBO = 128 B between core matrices along K, SBO = 1 KB between 8-row
// groups), two K-chunks of 32 in flight.  Inputs are rounded to TF32 (10-bit mantissa) on the way
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
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < TC_WAIT; ++it) {
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
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * stage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * stage + 16);
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
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[1])), "r"(1));
  }
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
  bool ok = true;
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
    const int j0 = c * TC_KC;
    if (flip) {
      // warp w stages lines 16w..16w+15; one load instruction covers 8 lines x 4 consecutive j
      // (8 sectors) and its shared-memory stores hit 32 distinct banks
#pragma unroll 4
      for (int i = 0; i < 16; ++i) {
        const int row = 16 * warp + 8 * (i & 1) + (lane >> 2), k = 4 * (i >> 1) + (lane & 3), j = j0 + k;
        const int64_t Lr = L0 + row;
        const float v = (Lr < a.nlines && j < n) ? x[Lr * n + j] : 0.0f;
        *reinterpret_cast<float*>(sx + cm_off(row, k)) = to_tf32(v);
      }
    } else {
      // half of this thread's line: 16 values, as four 16-byte rows of core matrices
      float v[TC_KC / 2];
#pragma unroll
      for (int jj = 0; jj < TC_KC / 2; ++jj) {
        const int j = j0 + 16 * hf + jj;
        v[jj] = (live && j < n) ? x[base + (int64_t)j * jstep] : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < TC_KC / 8; ++q) {
        const float4 w = make_float4(to_tf32(v[4 * q]), to_tf32(v[4 * q + 1]), to_tf32(v[4 * q + 2]),
                                     to_tf32(v[4 * q + 3]));
        *reinterpret_cast<float4*>(sx + cm_off(ln, 16 * hf + 4 * q)) = w;
      }
    }
    {   // the chunk's block of S, stored in the shared-memory layout: a straight 16-byte copy
      const float4* src = reinterpret_cast<const float4*>(a.S + (int64_t)c * N * TC_KC);
      float4* dst = reinterpret_cast<float4*>(ss);
      for (int i = tid; i < N * TC_KC / 4; i += TC_THREADS) dst[i] = __ldg(&src[i]);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
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
  }
  // the last commit tracks every MMA of the CTA
  if (ok) ok = __syncthreads_and(bar_wait(smem_u32(&bars[(C - 1) & 1]), ((C - 1) >> 1) & 1) ? 1 : 0) != 0;
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 1);
    // give the MMAs in flight a further bounded wait before the accumulators are released
    bar_wait(smem_u32(&bars[(C - 1) & 1]), ((C - 1) >> 1) & 1);
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

size_t tc_smem_bytes(int N) { return 2 * (size_t)(TC_M * TC_KC * 4 + N * TC_KC * 4) + 64; }

cudaError_t init_tc_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_mode<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes(256));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_mode<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes(256));
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
