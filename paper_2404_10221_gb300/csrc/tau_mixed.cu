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
#include "tau_group.cuh"

namespace tau {

constexpr int MX_THREADS = 256;

struct RresArgs {
  const int* flag;
  const double* E;
  const double* u;
  const double* src;   // k_rres_line: source of the factor
  double* y;           // save / add: y; line: destination of the factor
  const double* r;
  double* b;
  const double* fdt;
  int64_t n;
  unsigned stride, nk;
  double bd, bo;
  int fin, r_df;
  int mode;            // 0 save: y = E∘u; 1 add: y += E∘u; 2 one factor of B (line)
  int pad;
};

// mode 0: y = E_m∘u (before the fields of the new step overwrite E); mode 1: y += E_{m+1}∘u;
// mode 2: one factor of B = B_{d-1} ⊗ ... ⊗ B_0 along the dimension with element stride `stride`
// and length nk: y = bd src + bo (src at the two neighbours along that dimension; zero outside).
// The last factor (fin) instead writes b = B y + r - b + Fdt, r stored in FP64 or (r_df) as
// double-float pairs.  Line indices are unsigned 32-bit (n_tot <= 2^31, so a grid-stride index
// stays below 2^32).
__device__ __forceinline__ void rres_run(const RresArgs& A, VB vb) {
  if (!*A.flag) return;
  if (A.mode == 0 || A.mode == 1) {
    for (int64_t i = vb.bid * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)vb.nb * blockDim.x)
      A.y[i] = A.mode == 0 ? A.E[i] * A.u[i] : fma(A.E[i], A.u[i], A.y[i]);
    return;
  }
  const unsigned n = (unsigned)A.n;
  for (unsigned i = vb.bid * blockDim.x + threadIdx.x; i < n; i += (unsigned)vb.nb * blockDim.x) {
    const unsigned ik = (i / A.stride) % A.nk;
    double v = A.bd * A.src[i];
    if (ik > 0) v = fma(A.bo, A.src[i - A.stride], v);
    if (ik + 1 < A.nk) v = fma(A.bo, A.src[i + A.stride], v);
    if (A.fin)
      A.b[i] = v + (A.r_df ? to_d(reinterpret_cast<const df64*>(A.r)[i]) : A.r[i]) - A.b[i] + A.fdt[i];
    else
      A.y[i] = v;
  }
}

struct RresBody {
  using Args = RresArgs;
  static constexpr int kThreads = MX_THREADS, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { rres_run(a, vb); }
};

__global__ void k_rres(const RresArgs A) { rres_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }

struct FlagArgs {
  int* flag;
  int v;
  int pad;
};
__device__ __forceinline__ void set_flag_run(const FlagArgs& A, VB) {
  if (threadIdx.x == 0) *A.flag = A.v;
}
struct FlagBody {
  using Args = FlagArgs;
  static constexpr int kThreads = 32, kCtas = 1;
  static __device__ __forceinline__ void run(const Args& a, VB vb) { set_flag_run(a, vb); }
};
__global__ void k_set_flag(const FlagArgs A) { set_flag_run(A, VB{(int)blockIdx.x, (int)gridDim.x}); }

static unsigned mx_blocks(int64_t n) {
  const int64_t b = (n + MX_THREADS - 1) / MX_THREADS;
  return (unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

static cudaError_t rres_launch(const RresArgs& a, cudaStream_t st) {
  if (tl_rec) return record_launch<RresBody>(a, mx_blocks(a.n), MX_THREADS, 0);
  k_rres<<<mx_blocks(a.n), MX_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rres_save(const int* flag, const double* E, const double* u, double* y, int64_t n,
                             cudaStream_t st) {
  RresArgs a{};
  a.flag = flag;
  a.E = E;
  a.u = u;
  a.y = y;
  a.n = n;
  a.mode = 0;
  return rres_launch(a, st);
}

cudaError_t launch_rres_rhs(const int* flag, int d, const int* nn, const double* bd, const double* bo,
                            const double* E, const double* u, double* y, double* y2, const double* r, int r_df,
                            double* b, const double* fdt, int64_t n, cudaStream_t st) {
  RresArgs a{};
  a.flag = flag;
  a.E = E;
  a.u = u;
  a.y = y;
  a.n = n;
  a.mode = 1;
  cudaError_t e = rres_launch(a, st);
  if (e != cudaSuccess) return e;
  // B one dimension at a time, y -> y2 -> y -> ..., the last factor combining into b
  double* bufs[2] = {y, y2};
  int64_t stride = 1;
  for (int ax = 0; ax < d; ++ax) {
    RresArgs l{};
    l.flag = flag;
    l.src = bufs[ax & 1];
    l.y = bufs[(ax + 1) & 1];
    l.n = n;
    l.stride = (unsigned)stride;
    l.nk = (unsigned)nn[ax];
    l.bd = bd[ax];
    l.bo = bo[ax];
    l.fin = ax == d - 1;
    l.r = r;
    l.r_df = r_df;
    l.b = b;
    l.fdt = fdt;
    l.mode = 2;
    e = rres_launch(l, st);
    if (e != cudaSuccess) return e;
    stride *= nn[ax];
  }
  return cudaSuccess;
}

cudaError_t launch_set_flag(int* flag, int v, cudaStream_t st) {
  const FlagArgs a{flag, v, 0};
  if (tl_rec) return record_launch<FlagBody>(a, 1, 32, 0);
  k_set_flag<<<1, 32, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tau
