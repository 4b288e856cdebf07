// Grouped execution of many problems' kernels as one launch (batched and served forms).
//
// A kernel body runs on virtual blocks VB{bid, nb}: in a plain launch (blockIdx.x, gridDim.x); in a
// grouped launch the grid is the concatenation of every problem's grid, problem i owning blocks
// [start[i], start[i+1]), and each block runs the body with problem i's arguments and its index in
// that range.  Problems keep their own device state (Arnoldi index, stop flags, reduction tickets),
// so a grouped launch computes exactly what the per-problem launches compute.
//
// While a recorder is installed (tl_rec), the launch functions append their launch (grouped
// kernel, argument bytes, grid, block, shared memory) instead of launching; tau_batch merges the
// records of the problems of a group position by position into grouped launches.
#pragma once

#include "tau_internal.cuh"

namespace tau {

// Blocks of problem i: [start[i], start[i+1]).  The block's problem is the last i with
// start[i] <= blockIdx.x (problems with no blocks are skipped), its arguments are copied to shared
// memory once, and the body runs on them.
template <typename B>
__global__ void __launch_bounds__(B::kThreads, B::kCtas)
    k_grouped(const typename B::Args* __restrict__ args, const int* __restrict__ start, int n) {
  using A = typename B::Args;
  static_assert(sizeof(A) % 4 == 0, "argument blocks are copied in 4-byte words");
  __shared__ int s_i;
  __shared__ __align__(16) unsigned char s_args[sizeof(A)];
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;
    const int b = (int)blockIdx.x;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&start[mid]) <= b) lo = mid;
      else hi = mid - 1;
    }
    s_i = lo;
  }
  __syncthreads();
  const int i = s_i;
  const unsigned* src = reinterpret_cast<const unsigned*>(args + i);
  unsigned* dst = reinterpret_cast<unsigned*>(s_args);
  for (int w = threadIdx.x; w < (int)(sizeof(A) / 4); w += blockDim.x) dst[w] = __ldg(&src[w]);
  const int b0 = __ldg(&start[i]), b1 = __ldg(&start[i + 1]);
  __syncthreads();
  B::run(*reinterpret_cast<const A*>(s_args), VB{(int)blockIdx.x - b0, b1 - b0});
}

// Record a launch of body B (a recorder must be installed).
template <typename B>
cudaError_t record_launch(const typename B::Args& a, unsigned grid, unsigned block, size_t smem) {
  LaunchRec r;
  r.fn = reinterpret_cast<const void*>(&k_grouped<B>);
  r.args.assign(reinterpret_cast<const unsigned char*>(&a), reinterpret_cast<const unsigned char*>(&a) + sizeof(a));
  r.grid = grid;
  r.block = block;
  r.smem = smem;
  r.kthreads = B::kThreads;
  tl_rec->push_back(std::move(r));
  return cudaSuccess;
}

// Graph condition of a device-controlled loop.  use_cond 1: this problem's own handle; 2: the
// handle of a group, set by the last of its n problems to report (to 1 when any of them continues).
// Every problem of a group reports exactly once per launch of the reporting kernel.
__device__ __forceinline__ void report_cond(int use_cond, GroupCtl* gc, bool cont, cudaGraphConditionalHandle h1,
                                            cudaGraphConditionalHandle h2, bool two) {
  if (use_cond == 1) {
    cudaGraphSetConditional(h1, cont ? 1 : 0);
    if (two) cudaGraphSetConditional(h2, cont ? 1 : 0);
  } else if (use_cond == 2) {
    if (cont) atomicOr(&gc->any, 1);
    __threadfence();
    if (atomicAdd(&gc->ticket, 1u) == (unsigned)gc->n - 1u) {
      const int any = atomicExch(&gc->any, 0);
      gc->ticket = 0u;
      __threadfence();
      cudaGraphSetConditional(h1, any ? 1 : 0);
      if (two) cudaGraphSetConditional(h2, any ? 1 : 0);
    }
  }
}

}  // namespace tau
