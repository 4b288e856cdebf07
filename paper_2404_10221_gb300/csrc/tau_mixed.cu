// Right-hand side of the next step from the last residual (mixed-precision form).
//
// The refinement of step m ends with r = b - A_m x computed in FP64 for its final iterate x =
// u^(m+1) (the loop stops right after a residual; Eq. (tls): A_m = B E_m + S).  Since
// A_m x = B(E_m∘x) + S x, the right-hand side of step m+1,
//     b' = (B E_{m+1} - S) x + dt F_{m+1},
// equals B((E_m + E_{m+1})∘x) + r - b + dt F_{m+1}: one application of the tridiagonal product
// B = ⊗ B_{alpha_i} (d three-point passes, one per factor) in place of the three FP64 Toeplitz line
// passes.  A device
// flag says whether r belongs to the current solution (set at the end of every step, cleared when
// the caller replaces the solution); the line passes of the usual right-hand side skip themselves
// when it is set, these kernels return at once when it is not.
#include "tau_internal.cuh"

namespace tau {

constexpr int MX_THREADS = 256;

// y = E_m∘u (before the fields of the new step overwrite E)
__global__ void k_rres_save(const int* __restrict__ flag, const double* __restrict__ E, const double* __restrict__ u,
                            double* y, int64_t n) {
  if (!*flag) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = E[i] * u[i];
}

// y += E_{m+1}∘u
__global__ void k_rres_add(const int* __restrict__ flag, const double* __restrict__ E, const double* __restrict__ u,
                           double* y, int64_t n) {
  if (!*flag) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(E[i], u[i], y[i]);
}

// One factor of B = B_{d-1} ⊗ ... ⊗ B_0 along the dimension with element stride `stride` and
// length nk: dst = bd src + bo (src at the two neighbours along that dimension; zero outside).  The
// last factor (fin) instead writes b = B y + r - b + Fdt, r stored in FP64 or (r_df) as double-float
// pairs.  Indices are unsigned 32-bit (n_tot <= 2^31, so a grid-stride index stays below 2^32).
__global__ void k_rres_line(const int* __restrict__ flag, const double* __restrict__ src, double* dst, unsigned n,
                            unsigned stride, unsigned nk, double bd, double bo, int fin,
                            const double* __restrict__ r, int r_df, double* b, const double* __restrict__ fdt) {
  if (!*flag) return;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned ik = (i / stride) % nk;
    double v = bd * src[i];
    if (ik > 0) v = fma(bo, src[i - stride], v);
    if (ik + 1 < nk) v = fma(bo, src[i + stride], v);
    if (fin)
      b[i] = v + (r_df ? to_d(reinterpret_cast<const df64*>(r)[i]) : r[i]) - b[i] + fdt[i];
    else
      dst[i] = v;
  }
}

__global__ void k_set_flag(int* flag, int v) { *flag = v; }

static unsigned mx_blocks(int64_t n) {
  const int64_t b = (n + MX_THREADS - 1) / MX_THREADS;
  return (unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

cudaError_t launch_rres_save(const int* flag, const double* E, const double* u, double* y, int64_t n,
                             cudaStream_t st) {
  k_rres_save<<<mx_blocks(n), MX_THREADS, 0, st>>>(flag, E, u, y, n);
  return cudaGetLastError();
}

cudaError_t launch_rres_rhs(const int* flag, int d, const int* nn, const double* bd, const double* bo,
                            const double* E, const double* u, double* y, double* y2, const double* r, int r_df,
                            double* b, const double* fdt, int64_t n, cudaStream_t st) {
  k_rres_add<<<mx_blocks(n), MX_THREADS, 0, st>>>(flag, E, u, y, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // B one dimension at a time, y -> y2 -> y -> ..., the last factor combining into b
  double* bufs[2] = {y, y2};
  int64_t stride = 1;
  for (int ax = 0; ax < d; ++ax) {
    const int fin = ax == d - 1;
    k_rres_line<<<mx_blocks(n), MX_THREADS, 0, st>>>(flag, bufs[ax & 1], bufs[(ax + 1) & 1], (unsigned)n,
                                                       (unsigned)stride, (unsigned)nn[ax], bd[ax], bo[ax], fin, r, r_df,
                                                       b, fdt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stride *= nn[ax];
  }
  return cudaSuccess;
}

cudaError_t launch_set_flag(int* flag, int v, cudaStream_t st) {
  k_set_flag<<<1, 1, 0, st>>>(flag, v);
  return cudaGetLastError();
}

}  // namespace tau
