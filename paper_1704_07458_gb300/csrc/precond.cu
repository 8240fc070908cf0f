// Chebyshev polynomial preconditioner for the callback slot of the solver
// (Algorithm 1, Eq. 2: W = K^-1 R with "any preconditioner").
//
// K^-1 r is `degree` steps of the Chebyshev iteration for A w = r, started
// from w = 0, with the Jacobi splitting D = diag(A) and the spectral interval
// [lmin, lmax] of D^-1 A (Saad, Iterative Methods for Sparse Linear Systems,
// 2nd ed., Sec. 12.1.1, Algorithm 12.1):
//   theta = (lmax + lmin) / 2, delta = (lmax - lmin) / 2, sigma = theta / delta,
//   rho_0 = 1 / sigma,  d_0 = D^-1 r / theta,  w_1 = d_0,
//   for k = 1 .. degree-1:
//     z = D^-1 (r - A w_k),  rho_k = 1 / (2 sigma - rho_{k-1}),
//     d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) z,  w_{k+1} = w_k + d_k.
// w = p(D^-1 A) D^-1 r for a fixed polynomial p, positive on [lmin, lmax], so
// K^-1 = D^-1/2 p(D^-1/2 A D^-1/2) D^-1/2 is symmetric positive definite: a
// valid LOBPCG preconditioner.  Every step is this library's SpMM plus one
// fused elementwise kernel over the n x ncols block; no host work per call.
#include <algorithm>

#include "kernels.cuh"

struct lobpcg_chebyshev {
  int64_t n = 0, max_cols = 0, ld = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  double* dinv = nullptr;  // 1 / diag(A)
  double *w = nullptr, *d = nullptr, *aw = nullptr;  // n x ld work blocks
  int degree = 0;
  double lmin = 0.0, lmax = 0.0;
};

namespace lob {
namespace {

__global__ void cheb_dinv_kernel(int64_t n, const int32_t* __restrict__ rp,
                                 const int32_t* __restrict__ ci, const double* __restrict__ v,
                                 const double* __restrict__ diag, double* __restrict__ dinv) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double x = 0.0;
  if (diag) {
    x = diag[r];
  } else {
    for (int p = rp[r]; p < rp[r + 1]; ++p)
      if (ci[p] == r) x += v[p];
  }
  dinv[r] = x != 0.0 ? 1.0 / x : 1.0;
}

// first step: d = D^-1 r / theta, w = d
__global__ void cheb_first_kernel(int64_t n, int m, const double* __restrict__ R, int64_t ldr,
                                  const double* __restrict__ dinv, double inv_theta,
                                  double* __restrict__ d, double* __restrict__ w, int64_t ld) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  const int64_t r = e / m;
  const int c = (int)(e % m);
  const double v = R[r * ldr + c] * dinv[r] * inv_theta;
  d[r * ld + c] = v;
  w[r * ld + c] = v;
}

// later steps: z = D^-1 (r - A w), d = a d + b z, w += d; the last step
// writes w into the output W
__global__ void cheb_step_kernel(int64_t n, int m, const double* __restrict__ R, int64_t ldr,
                                 const double* __restrict__ aw, const double* __restrict__ dinv,
                                 double a, double b, double* __restrict__ d,
                                 double* __restrict__ w, int64_t ld, double* __restrict__ Wout,
                                 int64_t ldw) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  const int64_t r = e / m;
  const int c = (int)(e % m);
  const double z = (R[r * ldr + c] - aw[r * ld + c]) * dinv[r];
  const double dn = a * d[r * ld + c] + b * z;
  const double wn = w[r * ld + c] + dn;
  d[r * ld + c] = dn;
  w[r * ld + c] = wn;
  if (Wout) Wout[r * ldw + c] = wn;
}

__global__ void copy_rows_kernel(int64_t n, int m, const double* __restrict__ S, int64_t lds,
                                 double* __restrict__ D, int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  const int64_t r = e / m;
  const int c = (int)(e % m);
  D[r * ldd + c] = S[r * lds + c];
}

unsigned blocks_of(int64_t total) { return (unsigned)std::max<int64_t>(1, ceil_div(total, 256)); }

}  // namespace
}  // namespace lob

LOBPCG_EXPORT int lobpcg_chebyshev_create(lobpcg_chebyshev_t* out, int64_t n,
                                          const int32_t* rowptr, const int32_t* col,
                                          const double* val, const double* diag, int degree,
                                          double lmin, double lmax, int64_t max_cols) {
  if (!out) return LOBPCG_ERR_ARG;
  *out = nullptr;
  if (n <= 0 || !rowptr || !col || !val || degree < 1 || degree > 64 || !(lmin > 0.0) ||
      !(lmax > lmin) || max_cols <= 0)
    return LOBPCG_ERR_ARG;
  auto* c = new (std::nothrow) lobpcg_chebyshev();
  if (!c) return LOBPCG_ERR_OOM;
  c->n = n;
  c->max_cols = max_cols;
  c->ld = lob::round_up(max_cols, 8);
  c->rowptr = rowptr;
  c->col = col;
  c->val = val;
  c->degree = degree;
  c->lmin = lmin;
  c->lmax = lmax;
  const size_t blk = (size_t)n * c->ld * sizeof(double);
  if (cudaMalloc(&c->dinv, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->w, blk) != cudaSuccess || cudaMalloc(&c->d, blk) != cudaSuccess ||
      cudaMalloc(&c->aw, blk) != cudaSuccess) {
    cudaGetLastError();
    lobpcg_chebyshev_destroy(c);
    return LOBPCG_ERR_OOM;
  }
  lob::cheb_dinv_kernel<<<lob::blocks_of(n), 256>>>(n, rowptr, col, val, diag, c->dinv);
  ++lob::g_launches;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    lobpcg_chebyshev_destroy(c);
    return LOBPCG_ERR_CUDA;
  }
  *out = c;
  return LOBPCG_OK;
}

LOBPCG_EXPORT int lobpcg_chebyshev_apply(void* ctx, int64_t n, int64_t ncols, const double* R,
                                         int64_t ldr, double* W, int64_t ldw, void* stream) {
  auto* c = static_cast<lobpcg_chebyshev*>(ctx);
  if (!c || n != c->n || ncols < 0 || ncols > c->max_cols || ldr < ncols || ldw < ncols ||
      (ncols > 0 && (!R || !W)))
    return LOBPCG_ERR_ARG;
  if (ncols == 0) return LOBPCG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int m = (int)ncols;
  const double theta = 0.5 * (c->lmax + c->lmin), delta = 0.5 * (c->lmax - c->lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const unsigned nb = lob::blocks_of(n * m);
  lob::cheb_first_kernel<<<nb, 256, 0, st>>>(n, m, R, ldr, c->dinv, 1.0 / theta, c->d, c->w,
                                             c->ld);
  ++lob::g_launches;
  for (int k = 1; k < c->degree; ++k) {
    int rc = lob::spmm(st, n, c->rowptr, c->col, c->val, c->w, c->ld, m, c->aw, c->ld, nullptr,
                       nullptr, 0);
    if (rc) return rc;
    const double rho1 = 1.0 / (2.0 * sigma - rho);
    lob::cheb_step_kernel<<<nb, 256, 0, st>>>(n, m, R, ldr, c->aw, c->dinv, rho1 * rho,
                                              2.0 * rho1 / delta, c->d, c->w, c->ld,
                                              k + 1 == c->degree ? W : nullptr, ldw);
    ++lob::g_launches;
    rho = rho1;
  }
  if (c->degree == 1) {
    lob::copy_rows_kernel<<<nb, 256, 0, st>>>(n, m, c->w, c->ld, W, ldw);
    ++lob::g_launches;
  }
  return cudaPeekAtLastError() == cudaSuccess ? LOBPCG_OK : LOBPCG_ERR_CUDA;
}

LOBPCG_EXPORT void lobpcg_chebyshev_destroy(lobpcg_chebyshev_t c) {
  if (!c) return;
  cudaDeviceSynchronize();
  if (c->dinv) cudaFree(c->dinv);
  if (c->w) cudaFree(c->w);
  if (c->d) cudaFree(c->d);
  if (c->aw) cudaFree(c->aw);
  delete c;
}
