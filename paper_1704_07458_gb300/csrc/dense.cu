// Small dense layer: see dense.cuh.
#include <algorithm>
#include <cmath>
#include <cfloat>
#include <cstring>
#include <vector>

#include "dense.cuh"

namespace lob {

#define SOL_OK(expr)                                                   \
  do {                                                                 \
    if ((expr) != CUSOLVER_STATUS_SUCCESS) return LOBPCG_ERR_CUDA;     \
  } while (0)
#define BLAS_OK(expr)                                                  \
  do {                                                                 \
    if ((expr) != CUBLAS_STATUS_SUCCESS) return LOBPCG_ERR_CUDA;       \
  } while (0)

constexpr double kEps = 2.220446049250313e-16;  // 2^-52

// ------------------------------------------------------------------ kernels

// d_i = G_ii^-1/2, or 0 for a column of (numerically) zero norm.
__global__ void diag_inv_sqrt_kernel(int n, const double* G, int ldg, double* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double g = G[i + (int64_t)i * ldg];
  d[i] = g > DBL_MIN ? 1.0 / sqrt(g) : 0.0;
}

// M = diag(d) G diag(d), symmetrised from the lower triangle of G's product.
__global__ void scale_sym_kernel(int n, const double* G, int ldg, const double* d, double* M,
                                 int ldm) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  const double gij = G[i + (int64_t)j * ldg], gji = G[j + (int64_t)i * ldg];
  M[i + (int64_t)j * ldm] = d[i] * (0.5 * (gij + gji)) * d[j];
}

__global__ void copy_mat_kernel(int rows, int cols, const double* S, int lds, double* D,
                                int ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  D[i + (int64_t)j * ldd] = S[i + (int64_t)j * lds];
}

__global__ void scale_rows_kernel(int rows, int cols, const double* d, double* X, int ldx) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  X[i + (int64_t)j * ldx] *= d[i];
}

// T(:, t) = d .* Z(:, first + t) / sqrt(max(theta[first + t], floor)).
__global__ void svqb_t_kernel(int nu, int first, int nkeep, const double* d, const double* Z,
                              int ldz, const double* theta, double floor, double* T, int ldt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nu * nkeep) return;
  const int i = (int)(e % nu), t = (int)(e / nu);
  const double th = fmax(theta[first + t], floor);
  T[i + (int64_t)t * ldt] = d[i] * Z[i + (int64_t)(first + t) * ldz] / sqrt(th);
}

__global__ void assemble_kernel(int nx, int np, int nw, const double* theta, const double* PAP,
                                int ldpap, const double* GAw, const double* GBw, int ldgw,
                                double* SAS, double* SBS) {
  const int ns = nx + np + nw;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ns * ns) return;
  const int i = (int)(e % ns), j = (int)(e / ns);
  const int o = nx + np;
  double a = 0.0, b = (i == j) ? 1.0 : 0.0;
  if (j >= o) {
    a = GAw[i + (int64_t)(j - o) * ldgw];
    if (GBw) b = GBw[i + (int64_t)(j - o) * ldgw];
    if (i >= o) {  // W^T A W block: symmetrise
      a = 0.5 * (a + GAw[j + (int64_t)(i - o) * ldgw]);
      if (GBw) b = 0.5 * (b + GBw[j + (int64_t)(i - o) * ldgw]);
    }
  } else if (i >= o) {
    a = GAw[j + (int64_t)(i - o) * ldgw];
    if (GBw) b = GBw[j + (int64_t)(i - o) * ldgw];
  } else if (i < nx && j < nx) {
    a = (i == j) ? theta[i] : 0.0;
  } else if (i >= nx && j >= nx) {
    a = PAP[(i - nx) + (int64_t)(j - nx) * ldpap];
  }
  SAS[i + (int64_t)j * ns] = a;
  SBS[i + (int64_t)j * ns] = b;
}

__global__ void small_stats_kernel(const double* G, int rows, int cols, int ldg, int identity,
                                   const double* a, int na, const double* b, int nb,
                                   double* out) {
  __shared__ double red[3][256];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)rows * cols; e += blockDim.x) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    double g = G[i + (int64_t)j * ldg];
    if (identity && i == j) g -= 1.0;
    s0 = fma(g, g, s0);
  }
  for (int i = threadIdx.x; i < na; i += blockDim.x) s1 += a[i];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s2 += b[i];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  red[2][threadIdx.x] = s2;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int t = 0; t < 3; ++t) red[t][threadIdx.x] += red[t][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sqrt(red[0][0]);
    out[1] = red[1][0];
    out[2] = red[2][0];
  }
}

// cond(R) = sqrt(lambda_max(M) / lambda_min(M)) for M = R^T R (R upper, from
// potrf), estimated in one CTA: power iterations for lambda_max(M) and for
// lambda_max(M^-1) = 1/lambda_min(M), the latter through the two triangular
// solves with R.  FP32 arithmetic: the value only feeds the order-of-
// magnitude test cond(R)^-3 < tau_skip.  R is staged in shared memory when it
// fits (rstage != 0).  out[0] = cond estimate.
constexpr int kCondIters = 8;

__global__ void __launch_bounds__(256) cond_estimate_kernel(int n, const double* M, int ldm,
                                                            const double* R, int ldr, int rstage,
                                                            double* out) {
  extern __shared__ float sh[];
  float* x = sh;          // n
  float* y = sh + n;      // n
  float* Rs = sh + 2 * n; // n x n (column-major) when staged
  __shared__ float red[256];
  __shared__ float lmax_s;
  const int tid = threadIdx.x;
  auto block_sum = [&](float v) -> float {
    red[tid] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (tid < s) red[tid] += red[tid + s];
      __syncthreads();
    }
    const float r = red[0];
    __syncthreads();
    return r;
  };
  if (rstage)
    for (int64_t e = tid; e < (int64_t)n * n; e += 256) {
      const int i = (int)(e % n), j = (int)(e / n);
      Rs[e] = i <= j ? (float)R[i + (int64_t)j * ldr] : 0.f;
    }
  auto Rij = [&](int i, int j) -> float {
    return rstage ? Rs[i + (int64_t)j * n] : (float)R[i + (int64_t)j * ldr];
  };
  // lambda_max(M)
  for (int i = tid; i < n; i += 256) x[i] = 1.0f + 0.001f * (float)(i % 7);
  __syncthreads();
  float lam = 1.0f;
  for (int it = 0; it < kCondIters; ++it) {
    for (int i = tid; i < n; i += 256) {
      float s = 0.f;
      for (int j = 0; j < n; ++j) s += (float)M[i + (int64_t)j * ldm] * x[j];
      y[i] = s;
    }
    __syncthreads();
    float nx = 0.f, ny = 0.f, nn = 0.f;
    for (int i = tid; i < n; i += 256) {
      nx += x[i] * y[i];
      ny += y[i] * y[i];
      nn += x[i] * x[i];
    }
    const float xy = block_sum(nx), yy = block_sum(ny), xx = block_sum(nn);
    if (xx > 0.f) lam = fmaxf(lam, xy / xx);  // Rayleigh quotient
    const float inv = yy > 0.f ? rsqrtf(yy) : 0.f;
    for (int i = tid; i < n; i += 256) x[i] = y[i] * inv;
    __syncthreads();
  }
  if (tid == 0) lmax_s = lam;
  // lambda_max(M^-1) by x <- R^-1 R^-T x
  for (int i = tid; i < n; i += 256) x[i] = 1.0f - 0.002f * (float)(i % 5);
  __syncthreads();
  float mu = 0.f;
  bool bad = false;
  for (int it = 0; it < kCondIters && !bad; ++it) {
    // y = R^-T x: forward substitution, column-oriented (R^T lower)
    for (int i = tid; i < n; i += 256) y[i] = x[i];
    __syncthreads();
    for (int i = 0; i < n; ++i) {
      const float yi = y[i] / Rij(i, i);
      __syncthreads();
      for (int j = i + 1 + tid; j < n; j += 256) y[j] -= Rij(i, j) * yi;
      if (tid == 0) y[i] = yi;
      __syncthreads();
    }
    // x = R^-1 y: back substitution, column-oriented
    for (int i = n - 1; i >= 0; --i) {
      const float yi = y[i] / Rij(i, i);
      __syncthreads();
      for (int j = tid; j < i; j += 256) y[j] -= Rij(j, i) * yi;
      if (tid == 0) y[i] = yi;
      __syncthreads();
    }
    float a = 0.f, b = 0.f, c = 0.f;
    for (int i = tid; i < n; i += 256) {
      a += x[i] * y[i];
      b += y[i] * y[i];
      c += x[i] * x[i];
    }
    const float xy = block_sum(a), yy = block_sum(b), xx = block_sum(c);
    if (!(yy > 0.f) || !isfinite(yy)) bad = true;
    if (xx > 0.f) mu = fmaxf(mu, xy / xx);
    const float inv = (yy > 0.f && isfinite(yy)) ? rsqrtf(yy) : 0.f;
    for (int i = tid; i < n; i += 256) x[i] = y[i] * inv;
    __syncthreads();
  }
  if (tid == 0) {
    const double lmin = (bad || !(mu > 0.f)) ? 0.0 : 1.0 / (double)mu;
    out[0] = lmin > 0.0 ? sqrt((double)lmax_s / lmin) : INFINITY;
  }
}

// ------------------------------------------------------------------ helpers

static unsigned blocks_for(int64_t total) { return (unsigned)std::max<int64_t>(1, ceil_div(total, 256)); }

#define LAUNCH_OK(L)                                                  \
  do {                                                                \
    ++(L).launches;                                                   \
    ++g_launches;                                                     \
    if (cudaPeekAtLastError() != cudaSuccess) return LOBPCG_ERR_CUDA; \
  } while (0)

static int copy_mat(DenseLayer& L, int rows, int cols, const double* S, int lds, double* D,
                    int ldd) {
  if (rows <= 0 || cols <= 0) return LOBPCG_OK;
  copy_mat_kernel<<<blocks_for((int64_t)rows * cols), 256, 0, L.st>>>(rows, cols, S, lds, D, ldd);
  LAUNCH_OK(L);
  return LOBPCG_OK;
}

static int to_host(DenseLayer& L, double* dst, const void* src, size_t bytes) {
  LOB_CUDA_OK(cudaMemcpyAsync(L.host, src, bytes, cudaMemcpyDeviceToHost, L.st));
  LOB_CUDA_OK(cudaStreamSynchronize(L.st));
  memcpy(dst, L.host, bytes);
  return LOBPCG_OK;
}

// M = D G D with D = diag(G)^-1/2 (stored in L.d)
static int dscale(DenseLayer& L, int n, const double* G, int ldg, double* M, int ldm) {
  diag_inv_sqrt_kernel<<<blocks_for(n), 256, 0, L.st>>>(n, G, ldg, L.d);
  LAUNCH_OK(L);
  scale_sym_kernel<<<blocks_for((int64_t)n * n), 256, 0, L.st>>>(n, G, ldg, L.d, M, ldm);
  LAUNCH_OK(L);
  return LOBPCG_OK;
}

static int syevd(DenseLayer& L, bool vectors, int n, double* A, int lda) {
  SOL_OK(cusolverDnDsyevd(L.sol, vectors ? CUSOLVER_EIG_MODE_VECTOR : CUSOLVER_EIG_MODE_NOVECTOR,
                          CUBLAS_FILL_MODE_LOWER, n, A, lda, L.ev, L.work, L.lwork, L.info));
  return LOBPCG_OK;
}

// ------------------------------------------------------------------ API

int DenseLayer::init(cudaStream_t stream, int64_t n_max) {
  if (n_max <= nmax && sol) {
    st = stream;
    cusolverDnSetStream(sol, st);
    cublasSetStream(blas, st);
    return LOBPCG_OK;
  }
  release();
  st = stream;
  nmax = std::max<int64_t>(n_max, 8);
  SOL_OK(cusolverDnCreate(&sol));
  BLAS_OK(cublasCreate(&blas));
  SOL_OK(cusolverDnSetStream(sol, st));
  BLAS_OK(cublasSetStream(blas, st));
  const size_t mat = (size_t)nmax * nmax * sizeof(double);
  for (auto& a : A)
    if (cudaMalloc(&a, mat) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&ev, nmax * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&d, nmax * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&tau, nmax * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&scal, 16 * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&info, 4 * sizeof(int)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMallocHost(&host, (nmax + 64) * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  const int n = (int)nmax;
  int lw = 0, best = 0;
  SOL_OK(cusolverDnDsyevd_bufferSize(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                     A[0], n, ev, &lw));
  best = std::max(best, lw);
  SOL_OK(cusolverDnDpotrf_bufferSize(sol, CUBLAS_FILL_MODE_UPPER, n, A[0], n, &lw));
  best = std::max(best, lw);
  SOL_OK(cusolverDnDgeqrf_bufferSize(sol, n, n, A[0], n, &lw));
  best = std::max(best, lw);
  SOL_OK(cusolverDnDorgqr_bufferSize(sol, n, n, n, A[0], n, tau, &lw));
  best = std::max(best, lw);
  lwork = best;
  if (cudaMalloc(&work, (size_t)std::max(lwork, 1) * sizeof(double)) != cudaSuccess)
    return LOBPCG_ERR_OOM;
  return LOBPCG_OK;
}

void DenseLayer::release() {
  for (auto& a : A) {
    if (a) cudaFree(a);
    a = nullptr;
  }
  if (ev) cudaFree(ev);
  if (d) cudaFree(d);
  if (tau) cudaFree(tau);
  if (scal) cudaFree(scal);
  if (info) cudaFree(info);
  if (work) cudaFree(work);
  if (host) cudaFreeHost(host);
  ev = d = tau = scal = work = host = nullptr;
  info = nullptr;
  if (sol) cusolverDnDestroy(sol);
  if (blas) cublasDestroy(blas);
  sol = nullptr;
  blas = nullptr;
  nmax = 0;
}

int rr_initial(DenseLayer& L, const double* GA, const double* GB, int nx, double* C,
               double* theta, bool* breakdown) {
  *breakdown = false;
  double* MB = L.A[0];
  double* MA = L.A[1];
  double* Mc = L.A[2];
  const int ld = nx;
  int rc;
  if ((rc = dscale(L, nx, GB, nx, MB, ld))) return rc;
  scale_sym_kernel<<<blocks_for((int64_t)nx * nx), 256, 0, L.st>>>(nx, GA, nx, L.d, MA, ld);
  LAUNCH_OK(L);
  if ((rc = copy_mat(L, nx, nx, MB, ld, Mc, ld))) return rc;
  if ((rc = syevd(L, false, nx, Mc, ld))) return rc;
  SOL_OK(cusolverDnDpotrf(L.sol, CUBLAS_FILL_MODE_UPPER, nx, MB, ld, L.work, L.lwork, L.info));
  LOB_CUDA_OK(cudaMemcpyAsync(L.host, L.ev, nx * sizeof(double), cudaMemcpyDeviceToHost, L.st));
  LOB_CUDA_OK(cudaMemcpyAsync(L.host + nx, L.info, sizeof(int), cudaMemcpyDeviceToHost, L.st));
  LOB_CUDA_OK(cudaStreamSynchronize(L.st));
  int info;
  memcpy(&info, L.host + nx, sizeof(int));
  const double lo = L.host[0], hi = L.host[nx - 1];
  if (info != 0 || !(lo > nx * kEps * hi)) {
    *breakdown = true;
    return LOBPCG_OK;
  }
  const double one = 1.0;
  BLAS_OK(cublasDtrsm(L.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                      CUBLAS_DIAG_NON_UNIT, nx, nx, &one, MB, ld, MA, ld));
  BLAS_OK(cublasDtrsm(L.blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T,
                      CUBLAS_DIAG_NON_UNIT, nx, nx, &one, MB, ld, MA, ld));
  if ((rc = syevd(L, true, nx, MA, ld))) return rc;
  BLAS_OK(cublasDtrsm(L.blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                      CUBLAS_DIAG_NON_UNIT, nx, nx, &one, MB, ld, MA, ld));
  scale_rows_kernel<<<blocks_for((int64_t)nx * nx), 256, 0, L.st>>>(nx, nx, L.d, MA, ld);
  LAUNCH_OK(L);
  if ((rc = copy_mat(L, nx, nx, MA, ld, C, nx))) return rc;
  LOB_CUDA_OK(cudaMemcpyAsync(theta, L.ev, nx * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
  return LOBPCG_OK;
}

int rr_modified(DenseLayer& L, const double* SAS, const double* SBS, int ns, int nx, int nc,
                bool use_ortho, double tau_skip, bool* flip, double* condR, double* C,
                int* npn_out, double* theta, double* PAP) {
  *flip = false;
  *condR = 1.0;
  const int ld = ns;
  double* Rm = L.A[0];  // Cholesky factor
  double* H = L.A[1];   // projected matrix, then Z
  double* Tz = L.A[2];  // T Z
  double* M = L.A[3];   // Z_1perp^T Z_1(:, nc:nx), then Q
  double* Q2 = L.A[4];  // diag(theta_perp) Q
  const double one = 1.0, zero = 0.0;
  int rc;
  if (use_ortho) {
    if ((rc = copy_mat(L, ns, ns, SAS, ns, H, ld))) return rc;
    if ((rc = syevd(L, true, ns, H, ld))) return rc;
    if ((rc = copy_mat(L, ns, ns, H, ld, Tz, ld))) return rc;
  } else {
    if ((rc = dscale(L, ns, SBS, ns, Rm, ld))) return rc;
    scale_sym_kernel<<<blocks_for((int64_t)ns * ns), 256, 0, L.st>>>(ns, SAS, ns, L.d, H, ld);
    LAUNCH_OK(L);
    if ((rc = copy_mat(L, ns, ns, Rm, ld, Tz, ld))) return rc;
    SOL_OK(cusolverDnDpotrf(L.sol, CUBLAS_FILL_MODE_UPPER, ns, Rm, ld, L.work, L.lwork, L.info));
    LOB_CUDA_OK(cudaMemcpyAsync(L.host + 1, L.info, sizeof(int), cudaMemcpyDeviceToHost, L.st));
    LOB_CUDA_OK(cudaStreamSynchronize(L.st));
    int info;
    memcpy(&info, L.host + 1, sizeof(int));
    if (info != 0) {
      *flip = true;
      *condR = INFINITY;
      return LOBPCG_OK;
    }
    {
      // stage R in shared memory when it fits (227 KB per block)
      const size_t full = (size_t)(2 * ns + (size_t)ns * ns) * sizeof(float);
      const int rstage = full <= 200 * 1024 ? 1 : 0;
      const size_t bytes = rstage ? full : 2 * ns * sizeof(float);
      static bool configured = false;
      if (!configured) {
        LOB_CUDA_OK(cudaFuncSetAttribute(cond_estimate_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        configured = true;
      }
      cond_estimate_kernel<<<1, 256, bytes, L.st>>>(ns, Tz, ld, Rm, ld, rstage, L.scal);
      LAUNCH_OK(L);
    }
    double cr;
    if ((rc = to_host(L, &cr, L.scal, sizeof(double)))) return rc;
    *condR = cr;
    if (!(pow(*condR, -3.0) >= tau_skip)) {
      *flip = true;
      return LOBPCG_OK;
    }
    BLAS_OK(cublasDtrsm(L.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                        CUBLAS_DIAG_NON_UNIT, ns, ns, &one, Rm, ld, H, ld));
    BLAS_OK(cublasDtrsm(L.blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T,
                        CUBLAS_DIAG_NON_UNIT, ns, ns, &one, Rm, ld, H, ld));
    if ((rc = syevd(L, true, ns, H, ld))) return rc;
    if ((rc = copy_mat(L, ns, ns, H, ld, Tz, ld))) return rc;
    BLAS_OK(cublasDtrsm(L.blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                        CUBLAS_DIAG_NON_UNIT, ns, ns, &one, Rm, ld, Tz, ld));
    scale_rows_kernel<<<blocks_for((int64_t)ns * ns), 256, 0, L.st>>>(ns, ns, L.d, Tz, ld);
    LAUNCH_OK(L);
  }
  // C_p from the LQ form of Sec. 4.2 restricted to the unlocked columns.
  const int mrow = ns - nx, mcol = nx - nc;
  const int npn = std::min(mrow, mcol);
  if ((rc = copy_mat(L, ns, nx, Tz, ld, C, ns))) return rc;
  if (npn > 0) {
    BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_T, CUBLAS_OP_N, mrow, mcol, nx, &one,
                        H + (int64_t)nx * ld, ld, H + (int64_t)nc * ld, ld, &zero, M, ld));
    SOL_OK(cusolverDnDgeqrf(L.sol, mrow, mcol, M, ld, L.tau, L.work, L.lwork, L.info));
    SOL_OK(cusolverDnDorgqr(L.sol, mrow, npn, npn, M, ld, L.tau, L.work, L.lwork, L.info));
    BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_N, CUBLAS_OP_N, ns, npn, mrow, &one,
                        Tz + (int64_t)nx * ld, ld, M, ld, &zero, C + (int64_t)nx * ns, ns));
    if ((rc = copy_mat(L, mrow, npn, M, ld, Q2, ld))) return rc;
    scale_rows_kernel<<<blocks_for((int64_t)mrow * npn), 256, 0, L.st>>>(mrow, npn, L.ev + nx,
                                                                        Q2, ld);
    LAUNCH_OK(L);
    BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_T, CUBLAS_OP_N, npn, npn, mrow, &one, M, ld, Q2, ld,
                        &zero, PAP, npn));
  }
  LOB_CUDA_OK(cudaMemcpyAsync(theta, L.ev, nx * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
  *npn_out = npn;
  return LOBPCG_OK;
}

int svqb_transform(DenseLayer& L, const double* G, int nu, bool drop, double tau, double* T,
                   int* nkeep) {
  *nkeep = 0;
  if (nu <= 0) return LOBPCG_OK;
  double* Z = L.A[0];
  int rc;
  if ((rc = dscale(L, nu, G, nu, Z, nu))) return rc;
  if ((rc = syevd(L, true, nu, Z, nu))) return rc;
  std::vector<double> thv(nu);
  double* th = thv.data();
  if ((rc = to_host(L, th, L.ev, nu * sizeof(double)))) return rc;
  double mx = 0.0;
  for (int i = 0; i < nu; ++i) mx = std::max(mx, std::fabs(th[i]));
  if (!(mx > 0.0)) return LOBPCG_OK;
  int first = 0;
  double floor = -INFINITY;
  if (drop) {
    while (first < nu && !(th[first] > tau * mx)) ++first;
  } else {
    floor = tau * mx;
  }
  const int keep = nu - first;
  if (keep > 0) {
    svqb_t_kernel<<<blocks_for((int64_t)nu * keep), 256, 0, L.st>>>(nu, first, keep, L.d, Z, nu,
                                                                    L.ev, floor, T, nu);
    LAUNCH_OK(L);
  }
  *nkeep = keep;
  return LOBPCG_OK;
}

int assemble(DenseLayer& L, int nx, int np, int nw, const double* theta, const double* PAP,
             int ldpap, const double* GAw, const double* GBw, int ldgw, double* SAS,
             double* SBS) {
  const int ns = nx + np + nw;
  assemble_kernel<<<blocks_for((int64_t)ns * ns), 256, 0, L.st>>>(nx, np, nw, theta, PAP,
                                                                  std::max(ldpap, 1), GAw, GBw,
                                                                  ldgw, SAS, SBS);
  LAUNCH_OK(L);
  return LOBPCG_OK;
}

int small_stats(DenseLayer& L, const double* G, int rows, int cols, int ldg, bool identity,
                const double* a, int na, const double* b, int nb, double out[3]) {
  small_stats_kernel<<<1, 256, 0, L.st>>>(G, rows, cols, std::max(ldg, 1), identity ? 1 : 0, a,
                                          na, b, nb, L.scal);
  LAUNCH_OK(L);
  return to_host(L, out, L.scal, 3 * sizeof(double));
}

}  // namespace lob
