// Right-hand side of the next step from the last residual (mixed-precision form).
//
// The refinement of step m ends with r = b - A_m x computed in FP64 for its final iterate x =
// u^(m+1) (the loop stops right after a residual; Eq. (tls): A_m = B E_m + S).  Since
// A_m x = B(E_m∘x) + S x, the right-hand side of step m+1,
//     b' = (B E_{m+1} - S) x + dt F_{m+1},
// equals B((E_m + E_{m+1})∘x) + r - b + dt F_{m+1}: one application of the tridiagonal product
// B = ⊗ B_{alpha_i} (a 3^d-point stencil) in place of the three FP64 Toeplitz line passes.  A device
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

// b = B y + r - b + Fdt, B the d-level tridiagonal product (weights bd_i on the line, bo_i on the two
// neighbours, zero outside the grid)
__global__ void k_rres_rhs(const int* __restrict__ flag, int d, int n0, int n1, int n2, double bd0, double bo0,
                           double bd1, double bo1, double bd2, double bo2, const double* __restrict__ y,
                           const double* __restrict__ r, double* b, const double* __restrict__ fdt, int64_t n) {
  if (!*flag) return;
  const int64_t s1 = n0, s2 = (int64_t)n0 * n1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(i % n0);
    const int64_t q = i / n0;
    const int i1 = d > 1 ? (int)(q % n1) : 0;
    const int i2 = d > 2 ? (int)(q / n1) : 0;
    double acc = 0.0;
    for (int o2 = (d > 2 ? -1 : 0); o2 <= (d > 2 ? 1 : 0); ++o2) {
      const int j2 = i2 + o2;
      if (j2 < 0 || (d > 2 && j2 >= n2)) continue;
      const double w2 = d > 2 ? (o2 == 0 ? bd2 : bo2) : 1.0;
      for (int o1 = (d > 1 ? -1 : 0); o1 <= (d > 1 ? 1 : 0); ++o1) {
        const int j1 = i1 + o1;
        if (j1 < 0 || (d > 1 && j1 >= n1)) continue;
        const double w21 = w2 * (d > 1 ? (o1 == 0 ? bd1 : bo1) : 1.0);
        const int64_t row = (int64_t)o2 * s2 + (int64_t)o1 * s1;
        double line = bd0 * y[i + row];
        if (i0 > 0) line = fma(bo0, y[i + row - 1], line);
        if (i0 + 1 < n0) line = fma(bo0, y[i + row + 1], line);
        acc = fma(w21, line, acc);
      }
    }
    b[i] = acc + r[i] - b[i] + fdt[i];
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
                            const double* E, const double* u, double* y, const double* r, double* b,
                            const double* fdt, int64_t n, cudaStream_t st) {
  k_rres_add<<<mx_blocks(n), MX_THREADS, 0, st>>>(flag, E, u, y, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rres_rhs<<<mx_blocks(n), MX_THREADS, 0, st>>>(flag, d, nn[0], d > 1 ? nn[1] : 1, d > 2 ? nn[2] : 1, bd[0],
                                                    bo[0], d > 1 ? bd[1] : 1.0, d > 1 ? bo[1] : 0.0,
                                                    d > 2 ? bd[2] : 1.0, d > 2 ? bo[2] : 0.0, y, r, b, fdt, n);
  return cudaGetLastError();
}

cudaError_t launch_set_flag(int* flag, int v, cudaStream_t st) {
  k_set_flag<<<1, 1, 0, st>>>(flag, v);
  return cudaGetLastError();
}

}  // namespace tau
