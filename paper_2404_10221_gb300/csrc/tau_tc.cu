// Tensor-core (tcgen05, TF32) DST-I mode product for the FP32 τ solve of the mixed-precision form.
//
// The orthonormal DST-I along one dimension of length n <= 256 is a dense product with the
// symmetric sine matrix S (§3): for every grid line L, y_L[k] = sum_j S[k][j] x_L[j].  Its rows
// satisfy S[n-1-k][j] = (-1)^j S[k][j], so with E_k and O_k the sums over even and odd j,
// y[k] = E_k + O_k and y[n-1-k] = E_k - O_k: only the h = ceil(n/2) rows S_h are multiplied, the
// even and odd j into two accumulators (half the products and half the S traffic of the full
// matrix).  With 128 lines per CTA this is D(128 x Nh) = X(128 x K) S_h^T, K = n rounded up to 16:
// per K-chunk of 16 one tcgen05.mma.kind::tf32 over its 8 even j and one over its 8 odd j (M = 128,
// fp32 accumulators in tensor memory), the operands staged in shared memory in the 8-row x 16-byte
// core-matrix layout (K-major, no swizzle: LBO = 128 B between core matrices along K, SBO = 512 B
// between 8-row groups), a chunk's even j in slots 0-7 and its odd j in slots 8-15.  S_h is stored at
// setup in that layout chunk by chunk, and a chunk arrives by one tiled bulk copy (TMA, through a
// tensor map of the table seen as rows of 256 values).
//
// Pipeline: six shared-memory stages of one K-chunk each, nine warps.  Chunk c's line values are
// copied by the 256 threads of warps 0-7 with 4-byte asynchronous copies (cp.async, zero fill past
// the line's end) straight into their slots, and its block of S_h (stored at setup in that layout)
// by one tiled bulk copy (TMA, tensor map) issued by warp 8 on the stage's mbarrier; both are
// issued four chunks before the MMAs that read them.  A thread that sees its own copies of a chunk
// land rounds those values to TF32 in place (10-bit mantissa, nearest, ties away) and arrives on the
// stage's line barrier; warp 8 waits for both barriers of the chunk, issues its MMAs and commits
// them to the stage's release barrier, which the copies of the chunk six later wait for.  No
// block-wide barrier inside the K loop; every wait is bounded (mbarrier tests that suspend in
// hardware, a limited number of them).
//
// S is rounded to TF32 once at setup, so the product carries a relative error of order 1e-3: the
// flexible GMRES of the mixed form takes the result as its (variable) preconditioner, so this
// changes its iteration count, not the solution it converges to.  The epilogue reads both
// accumulators with tcgen05.ld (warp w owns lanes 32(w mod 4).., i.e. lines or outputs), forms
// E + O and E - O, optionally multiplies by a diagonal (the 1/mu of DST·(1/mu)·DST) and stores in
// place or out of place (each CTA reads all of its lines before it writes them).
#include "tau_internal.cuh"

#include <stdint.h>

namespace tau {

constexpr int TC_THREADS = 256;   // two warp groups: each TMEM lane quarter is read by two warps
constexpr int TD_THREADS = 288;   // DST: those two warp groups copy the lines, warp 8 issues the MMAs
constexpr int TC_M = 128;        // lines per CTA (accumulator rows = TMEM lanes)
constexpr int TC_KC = 16;        // K values per shared-memory stage (two MMAs of K = 8)
constexpr int TC_NST = 6;        // stages of the DST product
constexpr int TC_LA = 4;         // chunks copied ahead of the one whose MMAs are issued
constexpr int TC_WAIT = 4000000; // polls of an mbarrier before the kernel gives up

struct TcArgs {
  CUtensorMap tmS;       // S_h as a tensor of K-chunks (see TcTab::tmS)
  int n, ax, inner, N, Kp, nalloc;
  int64_t nlines;
  const float* S;        // per K-chunk c: the N x 16 block of S_h in the shared-memory core-matrix
                         // layout (N*16 floats at c*N*16), TF32-rounded, zero padded (read through tmS)
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

// byte offset of (row, k) in a K-major no-swizzle tile of 16 fp32 per row (8-row groups of 512 B)
__device__ __forceinline__ int cm16(int row, int k) {
  return (row >> 3) * 512 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
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

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, int limit = TC_WAIT) {
  for (int it = 0; it < limit; ++it) {
    if (bar_try(bar, parity)) return true;
    if (it > 64) __nanosleep(32);
  }
  return false;
}

// one test that may suspend the thread in hardware for up to TC_SUSPEND_NS while the phase is open
constexpr uint32_t TC_SUSPEND_NS = 10000;
constexpr int TC_WAIT_SUSPEND = 20000;   // such tests before a wait gives up (>= 0.2 s)
__device__ __forceinline__ bool bar_try_suspend(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity), "n"(TC_SUSPEND_NS)
      : "memory");
  return done != 0;
}

// bounded wait that also gives up as soon as another thread of the block has given up (*ab != 0)
__device__ __forceinline__ bool bar_wait_ab(uint32_t bar, uint32_t parity, const volatile int* ab) {
  for (int it = 0; it < TC_WAIT_SUSPEND; ++it) {
    if (bar_try_suspend(bar, parity)) return true;
    if (*ab) return false;
  }
  return false;
}

// Tiled bulk copy (TMA, tensor map in kernel-parameter space) of the box at coordinates (x, y) of a
// 2-D tensor into shared memory, completing on the mbarrier `bar` (which the caller armed with the
// box's byte count); x is 0 here, so the start is 16-byte aligned.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_init(uint32_t bar, int arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(arrivals));
}

__device__ __forceinline__ void bars_init(uint64_t* bars, int count) {
  for (int i = 0; i < count; ++i) bar_init(smem_u32(&bars[i]), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 4-byte asynchronous copy from global to shared memory (cached in L1); valid = false writes zero
// and reads nothing (source size 0; src must still be a mapped address)
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int P> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(P) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <bool MUL>
__global__ void __launch_bounds__(TD_THREADS, 2) k_tc_mode(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  if ((a.g && a.g->done) || (a.skip && *a.skip)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.N, n = a.n, h = (n + 1) >> 1;
  // dimension 0 (lines contiguous): D[k][line] = S_h X^T (A = S_h, 128 rows k, B = the lines,
  // N = 128), so TMEM lanes run along k and the stores along each line coalesce; other dimensions
  // (lines interleaved): D[line][k] = X S_h^T (A = the lines, B = S_h with N rows), lanes run across
  // lines.  Two accumulators: even j (column 0) and odd j (column half), half = nalloc / 2.
  const bool flip = a.ax == 0;
  const uint32_t half = (uint32_t)a.nalloc >> 1;
  const int xt = TC_M * TC_KC * 4;         // line tile (bytes)
  const int sbytes = N * TC_KC * 4;        // S_h tile
  const int stage = xt + sbytes;           // a multiple of 1 KB
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + TC_NST * stage);
  // lfull[s]: every producer thread's line values of the stage's chunk are in place and rounded
  // (TC_THREADS arrivals); sfull[s]: the stage's S_h block landed (one arrival with its byte
  // count); empt[s]: the MMAs that read the stage are done (tcgen05.commit)
  uint64_t* lfull = bars;
  uint64_t* sfull = bars + TC_NST;
  uint64_t* empt = bars + 2 * TC_NST;
  volatile int* ab = reinterpret_cast<volatile int*>(bars + 3 * TC_NST);   // a wait gave up
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 3 * TC_NST) + 1;
  const int64_t L0 = (int64_t)blockIdx.x * TC_M;
  const float* x = a.in_sel ? a.in_base + (int64_t)(a.g->j + a.in_sel - 1) * a.vstride : a.in;
  float* y = a.out_sel ? a.out_base + (int64_t)(a.g->j + a.out_sel - 1) * a.vstride : a.out;
  // producers (warps 0-7), other dimensions: thread tid owns line L0 + (tid mod 128) (element j at
  // base + j*jstep) and copies the even (hf = 0) or odd (hf = 1) values of each chunk; in the
  // epilogue warp w reads TMEM lanes 32 (w mod 4).. and every other block of 16 accumulator
  // columns.  Dimension 0: warp w copies lines 16w..16w+15, 8 lines x 4 slots per instruction.
  // Warp 8 stages S_h and issues the MMAs.
  const int ln = tid & (TC_M - 1), hf = (tid >> 7) & 1;
  const int64_t L = L0 + ln;
  const bool live = L < a.nlines && warp < 8;
  int64_t base = 0, jstep = 1;
  if (live && !flip) {
    const int64_t sl = L / a.inner, b = L - sl * a.inner;
    base = sl * n * a.inner + b;
    jstep = a.inner;
  }
  if (tid == 0) {
    for (int s = 0; s < TC_NST; ++s) {
      bar_init(smem_u32(&lfull[s]), TC_THREADS);
      bar_init(smem_u32(&sfull[s]), 1);
      bar_init(smem_u32(&empt[s]), 1);
    }
    *ab = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
  const int C = a.Kp / TC_KC;
  const uint32_t sm0 = smem_u32(sm);
  bool ok = true;
  uint32_t s_pend = 0, s_par = 0;   // MMA thread: stages with an S_h copy not yet seen landed, its parity
  int lastc = -1;                   // MMA thread: last chunk whose MMAs were committed

  if (warp == 8) {
    if (lane == 0) {
      // kind::tf32: D f32 (bits 4-5 = 1), A and B tf32 (bits 7-9, 10-12 = 2), both K-major,
      // N >> 3 at bit 17, M >> 4 at bit 24
      const int nmma = flip ? TC_M : N;
      const uint32_t idesc =
          (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nmma >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
      auto stage_s = [&](int c) {
        const int s = c % TC_NST;
        const uint32_t sb = smem_u32(&sfull[s]);
        bar_expect_tx(sb, (uint32_t)sbytes);
        tma_load_2d(sm0 + (uint32_t)(s * stage + xt), &a.tmS, 0, c * (N >> 4), sb);
        s_pend |= 1u << s;
        s_par = (s_par & ~(1u << s)) | ((uint32_t)((c / TC_NST) & 1) << s);
      };
      for (int c = 0; c < C && c < TC_LA; ++c) stage_s(c);
      for (int c = 0; c < C; ++c) {
        // S_h of chunk c + TC_LA, once the MMAs of chunk c + TC_LA - TC_NST released its stage
        const int cn = c + TC_LA;
        if (cn < C) {
          if (cn >= TC_NST && !bar_wait_ab(smem_u32(&empt[cn % TC_NST]), ((cn / TC_NST) - 1) & 1, ab)) {
            ok = false;
            break;
          }
          stage_s(cn);
        }
        const int s = c % TC_NST;
        const uint32_t par = (uint32_t)((c / TC_NST) & 1);
        if (!bar_wait_ab(smem_u32(&lfull[s]), par, ab) || !bar_wait_ab(smem_u32(&sfull[s]), par, ab)) {
          ok = false;
          break;
        }
        s_pend &= ~(1u << s);
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sx = sm0 + (uint32_t)(s * stage), ss = sx + (uint32_t)xt;
        const uint32_t acc = c > 0 ? 1u : 0u;
        // K step 0 (even j) into the first accumulator, K step 1 (odd j) into the second
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const uint64_t dx = smem_desc(sx + 256 * q, 128, 512), ds = smem_desc(ss + 256 * q, 128, 512);
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + half * q),
              "l"(flip ? ds : dx), "l"(flip ? dx : ds), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&empt[s])));
        lastc = c;
      }
    }
    __syncwarp();
  } else {
    // this thread's copies: 8 per chunk, destinations fixed within the stage, sources stepping
    // along the lines
    uint32_t d0;             // shared-memory offset of the first slot within a stage
    const float* p0;         // source of the first value (chunk 0)
    const float* p1 = x;     // dimension 0: the second line's source
    bool v0 = false, v1 = false;
    int jo[4] = {0, 0, 0, 0};
    if (flip) {
      const int ra = 16 * warp + (lane >> 2), a4 = lane & 3;
      d0 = (uint32_t)((ra >> 3) * 512 + (ra & 7) * 16 + a4 * 4);   // row ra + 8: + 512; slot group g: + 128 g
      v0 = L0 + ra < a.nlines;
      v1 = L0 + ra + 8 < a.nlines;
      p0 = v0 ? x + (L0 + ra) * n : x;
      p1 = v1 ? x + (L0 + ra + 8) * n : x;
      // slot 4g + a4 holds j = 2(4g + a4) (g < 2) or 2(4g + a4 - 8) + 1 (g >= 2)
      jo[0] = 2 * a4;
      jo[1] = 2 * a4 + 8;
      jo[2] = 2 * a4 + 1;
      jo[3] = 2 * a4 + 9;
    } else {
      d0 = (uint32_t)cm16(ln, 8 * hf);   // slot 8 hf + m: + (m / 4) 128 + (m mod 4) 4
      p0 = live ? x + base + hf * jstep : x;
    }
    const int64_t js2 = 2 * jstep;
    auto copy_lines = [&](int c) {
      const uint32_t sx = sm0 + (uint32_t)((c % TC_NST) * stage) + d0;
      const int j0 = c * TC_KC;
      if (flip) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int j = j0 + jo[g];
          const bool vj = j < n;
          cp_async4(sx + 128 * g, (v0 && vj) ? p0 + j : x, v0 && vj);
          cp_async4(sx + 512 + 128 * g, (v1 && vj) ? p1 + j : x, v1 && vj);
        }
      } else {
        const float* q = p0 + (int64_t)j0 * jstep;
        const int rem = n - j0 - hf;   // values j0 + 2m + hf < n  <=>  2m < rem
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const bool v = live && 2 * m < rem;
          cp_async4(sx + (m >> 2) * 128 + (m & 3) * 4, v ? q : x, v);
          q += js2;
        }
      }
    };
    // round this thread's own (landed) values of chunk c to TF32 in place
    auto round_lines = [&](int c) {
      unsigned char* sx = sm + (c % TC_NST) * stage + d0;
      if (flip) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          float* pa = reinterpret_cast<float*>(sx + 128 * g);
          float* pb = reinterpret_cast<float*>(sx + 512 + 128 * g);
          *pa = to_tf32(*pa);
          *pb = to_tf32(*pb);
        }
      } else {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          float4* pv = reinterpret_cast<float4*>(sx + 128 * r);
          float4 v = *pv;
          v.x = to_tf32(v.x);
          v.y = to_tf32(v.y);
          v.z = to_tf32(v.z);
          v.w = to_tf32(v.w);
          *pv = v;
        }
      }
    };
    // tick t: copies of chunk t (once the MMAs of chunk t - TC_NST released its stage), then the
    // chunk t - TC_LA handed to the MMA warp
    for (int t = 0; t < C + TC_LA; ++t) {
      if (t < C) {
        if (t >= TC_NST && !bar_wait_ab(smem_u32(&empt[t % TC_NST]), ((t / TC_NST) - 1) & 1, ab)) {
          ok = false;
          break;
        }
        copy_lines(t);
      }
      cp_async_commit();   // (an empty group past the last chunk keeps the count of groups uniform)
      const int cf = t - TC_LA;
      if (cf < 0) continue;
      cp_async_wait<TC_LA>();   // this thread's copies of chunk cf have landed
      round_lines(cf);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
      bar_arrive(smem_u32(&lfull[cf % TC_NST]));
    }
  }
  if (!ok) *ab = 1;
  __syncthreads();
  ok = *ab == 0;
  // the last commit tracks every MMA of the CTA
  if (ok && !bar_wait_ab(smem_u32(&empt[(C - 1) % TC_NST]), ((C - 1) / TC_NST) & 1, ab)) *ab = 1;
  __syncthreads();
  ok = *ab == 0;
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 1);
    // the copies and MMAs still in flight get a further bounded wait before the shared memory and
    // the accumulators are released
    cp_async_wait_all();
    if (warp == 8 && lane == 0) {
      for (int s = 0; s < TC_NST; ++s)
        if (s_pend & (1u << s)) bar_wait(smem_u32(&sfull[s]), (s_par >> s) & 1u);
      if (lastc >= 0) bar_wait(smem_u32(&empt[lastc % TC_NST]), (uint32_t)((lastc / TC_NST) & 1));
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && warp < 8) {
    // y[k] = E_k + O_k and y[n-1-k] = E_k - O_k for k < h (S[n-1-k][j] = (-1)^j S[k][j]; the middle
    // row of an odd n is its own mirror and is stored once); groups of 8 accumulator columns
    const float* __restrict__ mul = a.mul;
    const int ncol = flip ? TC_M : N;
    for (int cc = 8 * hf; cc < ncol; cc += 16) {
      uint32_t ve[8], vo[8];
      const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cc;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(ve[0]), "=r"(ve[1]), "=r"(ve[2]), "=r"(ve[3]), "=r"(ve[4]), "=r"(ve[5]), "=r"(ve[6]),
                     "=r"(ve[7])
                   : "r"(taddr));
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(vo[0]), "=r"(vo[1]), "=r"(vo[2]), "=r"(vo[3]), "=r"(vo[4]), "=r"(vo[5]), "=r"(vo[6]),
                     "=r"(vo[7])
                   : "r"(taddr + half));
      float mp[8], mm[8];
      if (flip) {   // lane = k, columns = lines L0 + cc + q
        const int k = 32 * (warp & 3) + lane, km = n - 1 - k;
        const int64_t nrem = a.nlines - (L0 + cc);
        const int nq = k < h ? (nrem < 8 ? (int)nrem : 8) : 0;
        const bool mirror = km > k;
        float* yk = y + (L0 + cc) * n + k;
        if (MUL) {   // the factors' loads issued before the accumulators are waited for
          const float* mk = mul + (L0 + cc) * n + k;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            mp[q] = q < nq ? __ldg(mk + (int64_t)q * n) : 0.0f;
            mm[q] = q < nq && mirror ? __ldg(mk + (int64_t)q * n + (km - k)) : 0.0f;
          }
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (q < nq) {
            const float e = __uint_as_float(ve[q]), o = __uint_as_float(vo[q]);
            float yp = e + o, ym = e - o;
            if (MUL) {
              yp *= mp[q];
              ym *= mm[q];
            }
            yk[(int64_t)q * n] = yp;
            if (mirror) yk[(int64_t)q * n + (km - k)] = ym;
          }
        }
      } else {   // lane = line, columns = k
        const int kend = live ? min(cc + 8, h) : 0;
        if (MUL) {
          const float* mf = mul + base + (int64_t)cc * jstep;
          const float* mb = mul + base + (int64_t)(n - 1 - cc) * jstep;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int k = cc + q;
            mp[q] = k < kend ? __ldg(mf) : 0.0f;
            mm[q] = k < kend && n - 1 - k > k ? __ldg(mb) : 0.0f;
            mf += jstep;
            mb -= jstep;
          }
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float* yf = y + base + (int64_t)cc * jstep;
        float* yb = y + base + (int64_t)(n - 1 - cc) * jstep;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int k = cc + q;
          if (k < kend) {
            const float e = __uint_as_float(ve[q]), o = __uint_as_float(vo[q]);
            float yp = e + o, ym = e - o;
            if (MUL) {
              yp *= mp[q];
              ym *= mm[q];
            }
            *yf = yp;
            if (n - 1 - k > k) *yb = ym;
          }
          yf += jstep;
          yb -= jstep;
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
// two tiled bulk copies (TMA, tensor maps of the pre-arranged tables) on the stage's mbarrier.  The stencil reads a and c (neighbours
// included) from global memory in the epilogue, so the pass writes new channel buffers.
constexpr int TM_KC = 16;

struct TcMvArgs {
  CUtensorMap tmThi, tmTlo;   // T_hi, T_lo as tensors of K-chunks (see TcTab)
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

__global__ void __launch_bounds__(TC_THREADS) k_tc_mv(const __grid_constant__ TcMvArgs a) {
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
      tma_load_2d(smem_u32(sth), &a.tmThi, 0, c * (N >> 4), smem_u32(&bars[2 + s]));
      tma_load_2d(smem_u32(stl), &a.tmTlo, 0, c * (N >> 4), smem_u32(&bars[2 + s]));
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
  a.tmThi = t.tmThi;
  a.tmTlo = t.tmTlo;
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

// stages, then 3 TC_NST mbarriers, the give-up flag and the TMEM address slot
size_t tc_smem_bytes(int N) {
  static_assert(3 * TC_NST * 8 + 8 <= 256, "barrier area");
  return TC_NST * (size_t)(TC_M * TC_KC * 4 + N * TC_KC * 4) + 256;
}

cudaError_t init_tc_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_mode<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes(128));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tc_mode<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes(128));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_mv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tm_smem_bytes(256));
}

cudaError_t launch_tc_dst(const PassT<float>& p, const TcTab& t, const float* mul, bool from_out, cudaStream_t st) {
  TcArgs a{};
  a.tmS = t.tmS;
  a.n = t.n;
  a.ax = p.ax;
  a.inner = (int)p.inner;
  a.N = t.Nh;
  a.Kp = t.Kp16;
  a.nalloc = t.nalloc_h;
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
    k_tc_mode<true><<<grid, TD_THREADS, tc_smem_bytes(t.Nh), st>>>(a);
  else
    k_tc_mode<false><<<grid, TD_THREADS, tc_smem_bytes(t.Nh), st>>>(a);
  return cudaGetLastError();
}

}  // namespace tau
