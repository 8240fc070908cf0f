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

__global__ void set_identity_kernel(int n, double* A, int lda) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  A[i + (int64_t)j * lda] = i == j ? 1.0 : 0.0;
}

__global__ void set_zero_kernel(int rows, int cols, double* D, int ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  D[(e % rows) + (e / rows) * (int64_t)ldd] = 0.0;
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

// Projected pencil on S = [X, P, W] (ns = nx + np + nw): the columns from c0
// on come from Grams S^T (A S)(:, c0:) in GAw and S^T (B S)(:, c0:) in GBw
// (GBw == nullptr: S^T B S = I there), mirrored below the diagonal and
// symmetrised where both indices are >= c0; the rest from the identities
// (12)-(14): X^T A X = Theta, X^T B X = I, X^T A P = X^T B P = 0, P^T B P = I,
// P^T A P from Eq. (14).  c0 = nx + np: only the W columns are computed (the
// method's own pencil); c0 = nx or 0: the comparison variants and the
// explicit Rayleigh-Ritz.
__global__ void assemble_kernel(int nx, int np, int nw, int c0, const double* theta,
                                const double* PAP, int ldpap, const double* GAw,
                                const double* GBw, int ldgw, double* SAS, double* SBS) {
  const int ns = nx + np + nw;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ns * ns) return;
  const int i = (int)(e % ns), j = (int)(e / ns);
  double a = 0.0, b = (i == j) ? 1.0 : 0.0;
  if (j >= c0) {
    a = GAw[i + (int64_t)(j - c0) * ldgw];
    if (GBw) b = GBw[i + (int64_t)(j - c0) * ldgw];
    if (i >= c0) {  // both computed: symmetrise
      a = 0.5 * (a + GAw[j + (int64_t)(i - c0) * ldgw]);
      if (GBw) b = 0.5 * (b + GBw[j + (int64_t)(i - c0) * ldgw]);
    }
  } else if (i >= c0) {
    a = GAw[j + (int64_t)(i - c0) * ldgw];
    if (GBw) b = GBw[j + (int64_t)(i - c0) * ldgw];
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

// cond(R) = sqrt(lambda_max(M) lambda_max(R^-1 R^-T)) for M = R^T R, from
// power iterations with the explicit inverse Rinv (one CTA, matrix-vector
// products only: every product is parallel over rows or columns).  The value
// feeds the order-of-magnitude test cond(R)^-3 < tau_skip, so the iterations
// run in FP32 on FP64 data.  out[0] = cond estimate (inf when Rinv or M gives
// a non-finite or non-positive value).
constexpr int kCondIters = 8;
constexpr int kCondThreads = 1024;

__global__ void __launch_bounds__(kCondThreads) cond_estimate_kernel(int n, const double* M,
                                                                     int ldm, const double* Ri,
                                                                     int ldr, double* out) {
  extern __shared__ float sh[];
  float* x = sh;          // n
  float* y = sh + n;      // n
  float* z = sh + 2 * n;  // n
  __shared__ float red[3][32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kCondThreads / 32;
  auto block_sum3 = [&](float a, float b, float c, float& ra, float& rb, float& rc) {
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
      red[0][warp] = a;
      red[1][warp] = b;
      red[2][warp] = c;
    }
    __syncthreads();
    ra = rb = rc = 0.f;
    for (int w = 0; w < nw; ++w) {
      ra += red[0][w];
      rb += red[1][w];
      rc += red[2][w];
    }
    __syncthreads();
  };
  // column-oriented product: y_i = sum_j A(j, i) x_j (warp per column i)
  auto colprod = [&](const double* A, int lda, bool upper_only, const float* in, float* outv) {
    for (int i = warp; i < n; i += nw) {
      float s = 0.f;
      const int jmax = upper_only ? i + 1 : n;
      for (int j = lane; j < jmax; j += 32) s += (float)A[j + (int64_t)i * lda] * in[j];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) outv[i] = s;
    }
    __syncthreads();
  };
  // row-oriented product with the upper triangle: y_i = sum_{j >= i} A(i, j) x_j
  auto rowprod_upper = [&](const double* A, int lda, const float* in, float* outv) {
    for (int i = tid; i < n; i += kCondThreads) {
      float s = 0.f;
      for (int j = i; j < n; ++j) s += (float)A[i + (int64_t)j * lda] * in[j];
      outv[i] = s;
    }
    __syncthreads();
  };
  auto power = [&](int which) -> float {  // 0: M (symmetric), 1: Rinv Rinv^T
    for (int i = tid; i < n; i += kCondThreads) x[i] = 1.0f + 0.001f * (float)(i % 7);
    __syncthreads();
    float lam = 0.f;
    for (int it = 0; it < kCondIters; ++it) {
      float* res = y;
      if (which == 0) {
        colprod(M, ldm, false, x, y);
      } else {
        colprod(Ri, ldr, true, x, y);  // y = Rinv^T x (Rinv upper: column i has rows <= i)
        rowprod_upper(Ri, ldr, y, z);  // z = Rinv y
        res = z;
      }
      float a = 0.f, b = 0.f, c = 0.f;
      for (int i = tid; i < n; i += kCondThreads) {
        a += x[i] * res[i];
        b += res[i] * res[i];
        c += x[i] * x[i];
      }
      float xy, yy, xx;
      block_sum3(a, b, c, xy, yy, xx);
      if (!(yy > 0.f) || !isfinite(yy)) return INFINITY;
      if (xx > 0.f) lam = fmaxf(lam, xy / xx);
      const float inv = rsqrtf(yy);
      for (int i = tid; i < n; i += kCondThreads) x[i] = res[i] * inv;
      __syncthreads();
    }
    return lam;
  };
  const float lmax = power(0);
  const float imax = power(1);
  if (tid == 0)
    out[0] = (isfinite(lmax) && isfinite(imax) && lmax > 0.f && imax > 0.f)
                 ? sqrt((double)lmax * (double)imax)
                 : INFINITY;
}


// ------------------------------------------------------------ eigensolver
// Symmetric eigendecomposition of the small projected matrices, designed for
// a part whose FP64 rate is 1/64 of its FP32 rate: cuSOLVER's FP32 syevd gives
// X0 (about 1e-7 accurate); two steps of the refinement of Ogita and Aishima
// ("Iterative refinement for symmetric eigenvalue decomposition", Japan J.
// Indust. Appl. Math. 35, 2018) in FP64 GEMMs bring every eigenpair whose
// eigenvalue is separated by more than delta to FP64 accuracy; eigenvalues
// closer than delta form clusters whose FP64 block of X^T A X is
// diagonalised by Jacobi rotations; a Newton-Schulz step before that restores
// orthonormality to rounding level.  One host read (the Rayleigh quotients,
// delta) per call.
//
// One refinement step for X ~ eigenvectors of A (n x n, column-major):
//   G = X^T X, R = I - G, S = X^T A X, d_i = s_ii / g_ii,
//   delta = 2 (||S - diag(d)||_F + ||A||_F ||R||_F),
//   E_ij = (s_ij + d_j r_ij) / (d_j - d_i) if |d_i - d_j| > delta, else r_ij / 2,
//   X <- X + X E,
// from X' = X (I + E) with X'^T X' = I and X'^T A X' diagonal to first order
// (E + E^T = R, E^T D + D E = D - S off the diagonal).

constexpr int kMaxRefineSteps = 6;
constexpr int kRefBlocks = 64;
constexpr int kMaxRun = 32;  // cluster blocks up to this size: Jacobi in shared memory

// A <- (A + A^T) / 2 in place (threads of the strict lower triangle)
__global__ void symmetrize_kernel(int n, double* A, int lda) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  if (i <= j) return;
  const double v = 0.5 * (A[i + (int64_t)j * lda] + A[j + (int64_t)i * lda]);
  A[i + (int64_t)j * lda] = v;
  A[j + (int64_t)i * lda] = v;
}

__global__ void to_f32_kernel(int64_t total, const double* __restrict__ A, float* __restrict__ B) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < total) B[e] = (float)A[e];
}
__global__ void to_f64_kernel(int64_t total, const float* __restrict__ A, double* __restrict__ B) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < total) B[e] = (double)A[e];
}

// partial[b] = (||S - diag(d)||_F^2, ||R||_F^2, ||A||_F^2) over block b's elements
__global__ void __launch_bounds__(256) oa_norms_kernel(int n, const double* __restrict__ S,
                                                       const double* __restrict__ G,
                                                       const double* __restrict__ A, int lda,
                                                       double* __restrict__ partial) {
  __shared__ double red[3][256];
  double a = 0.0, b = 0.0, c = 0.0;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    const double s = S[e], g = G[e];
    const double aij = A[i + (int64_t)j * lda];
    if (i == j) {
      const double d = g != 0.0 ? s / g : s;
      a = fma(s - d, s - d, a);
      b = fma(1.0 - g, 1.0 - g, b);
    } else {
      a = fma(s, s, a);
      b = fma(g, g, b);
    }
    c = fma(aij, aij, c);
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int t = 0; t < 3; ++t) red[t][threadIdx.x] += red[t][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int t = 0; t < 3; ++t) partial[blockIdx.x * 3 + t] = red[t][0];
}

// E from S, G and delta (every block reduces the partials itself); block 0
// stores delta and ||A||_F.
__global__ void __launch_bounds__(256) oa_update_kernel(int n, const double* __restrict__ S,
                                                        const double* __restrict__ G,
                                                        const double* __restrict__ partial,
                                                        int nparts, double* __restrict__ E,
                                                        double* __restrict__ delta_out) {
  __shared__ double dl;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int p = 0; p < nparts; ++p) {
      a += partial[3 * p];
      b += partial[3 * p + 1];
      c += partial[3 * p + 2];
    }
    dl = 2.0 * (sqrt(a) + sqrt(c) * sqrt(b));
    if (blockIdx.x == 0) {
      delta_out[0] = dl;
      delta_out[1] = sqrt(c);
    }
  }
  __syncthreads();
  const double delta = dl;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    const double g = G[e];
    double out;
    if (i == j) {
      out = 0.5 * (1.0 - g);
    } else {
      const double gi = G[i + (int64_t)i * n], gj = G[j + (int64_t)j * n];
      const double di = S[i + (int64_t)i * n] / gi, dj = S[j + (int64_t)j * n] / gj;
      const double r = -g;
      if (fabs(di - dj) > delta)
        out = (S[e] + dj * r) / (dj - di);
      else
        out = 0.5 * r;
    }
    E[e] = out;
  }
}

// G <- 3/2 I - 1/2 G: X (3/2 I - 1/2 X^T X) squares the orthogonality error
// of X (one Newton-Schulz step towards the orthogonal polar factor)
__global__ void newton_schulz_kernel(int n, double* G) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  G[e] = (i == j ? 1.5 : 0.0) - 0.5 * G[e];
}

// out = max_i sqrt(sum_{j : runid[j] != runid[i]} S_ij^2) (non-negative
// doubles order like their bit patterns, so atomicMax on the bits is a max)
__global__ void offrun_check_kernel(int n, const double* __restrict__ S,
                                    const int* __restrict__ runid,
                                    unsigned long long* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int ri = runid[i];
  double acc = 0.0;
  for (int j = 0; j < n; ++j) {
    if (runid[j] == ri) continue;
    const double v = S[i + (int64_t)j * n];
    acc = fma(v, v, acc);
  }
  const double r = sqrt(acc);
  atomicMax(out, (unsigned long long)__double_as_longlong(isfinite(r) ? r : INFINITY));
}

__global__ void diag_extract_kernel(int n, const double* __restrict__ S, const double* delta,
                                    double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = S[i + (int64_t)i * n];
  if (i == n) out[n] = *delta;
}

// Xo(:, k) = X(:, perm[k]); lam[k] = S(perm[k], perm[k])
__global__ void permute_cols_kernel(int n, const double* __restrict__ X,
                                    const double* __restrict__ S, const int* __restrict__ perm,
                                    double* __restrict__ Xo, int ldo, double* __restrict__ lam) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int r = (int)(e % n), k = (int)(e / n);
  const int p = perm[k];
  Xo[r + (int64_t)k * ldo] = X[r + (int64_t)p * n];
  if (r == 0) lam[k] = S[p + (int64_t)p * n];
}

// One block per cluster run [a, a + m) of the permuted order: cyclic Jacobi on
// the FP64 block S(perm[a + i], perm[a + j]) by one warp, eigenvalues sorted
// ascending, then Xo(:, a : a + m) <- Xo(:, a : a + m) Q by all threads.
__global__ void __launch_bounds__(256) cluster_jacobi_kernel(int n, const double* __restrict__ S,
                                                             const int* __restrict__ perm,
                                                             const int* __restrict__ runs,
                                                             double* __restrict__ Xo, int ldo,
                                                             double* __restrict__ lam) {
  __shared__ double M[kMaxRun][kMaxRun + 1], Q[kMaxRun][kMaxRun + 1];
  __shared__ double ev[kMaxRun];
  __shared__ int order[kMaxRun];
  const int a = runs[2 * blockIdx.x], m = runs[2 * blockIdx.x + 1];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e % m, j = e / m;
    const double sij = S[perm[a + i] + (int64_t)perm[a + j] * n];
    const double sji = S[perm[a + j] + (int64_t)perm[a + i] * n];
    M[i][j] = 0.5 * (sij + sji);
    Q[i][j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid < 32) {
    for (int sweep = 0; sweep < 30; ++sweep) {
      double off = 0.0, tot = 0.0;
      for (int e = lane; e < m * m; e += 32) {
        const int i = e % m, j = e / m;
        const double v = M[i][j] * M[i][j];
        tot += v;
        if (i != j) off += v;
      }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
      }
      if (!(off > 1e-30 * tot)) break;
      for (int p = 0; p < m - 1; ++p)
        for (int q = p + 1; q < m; ++q) {
          const double apq = M[p][q];
          if (apq == 0.0) continue;
          // rotation zeroing M[p][q] (Golub & Van Loan, Sec. 8.5.2)
          const double tau = (M[q][q] - M[p][p]) / (2.0 * apq);
          // hypot(1, tau): no overflow of tau^2 for tiny a_pq (small-angle t = 1/(2 tau))
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
          const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
          __syncwarp();
          for (int k = lane; k < m; k += 32) {  // columns p, q
            const double mkp = M[k][p], mkq = M[k][q];
            M[k][p] = c * mkp - s * mkq;
            M[k][q] = s * mkp + c * mkq;
            const double qkp = Q[k][p], qkq = Q[k][q];
            Q[k][p] = c * qkp - s * qkq;
            Q[k][q] = s * qkp + c * qkq;
          }
          __syncwarp();
          for (int k = lane; k < m; k += 32) {  // rows p, q
            const double mpk = M[p][k], mqk = M[q][k];
            M[p][k] = c * mpk - s * mqk;
            M[q][k] = s * mpk + c * mqk;
          }
          __syncwarp();
        }
    }
    if (lane == 0) {  // ascending order of the eigenvalues (insertion sort, m <= 32)
      for (int i = 0; i < m; ++i) {
        ev[i] = M[i][i];
        order[i] = i;
      }
      for (int i = 1; i < m; ++i)
        for (int j = i; j > 0 && ev[order[j]] < ev[order[j - 1]]; --j) {
          const int t = order[j];
          order[j] = order[j - 1];
          order[j - 1] = t;
        }
    }
  }
  __syncthreads();
  for (int i = tid; i < m; i += blockDim.x) lam[a + i] = ev[order[i]];
  for (int r = tid; r < n; r += blockDim.x) {
    double x[kMaxRun];
    for (int j = 0; j < m; ++j) x[j] = Xo[r + (int64_t)(a + j) * ldo];
    for (int i = 0; i < m; ++i) {
      const int c = order[i];
      double v = 0.0;
      for (int j = 0; j < m; ++j) v = fma(x[j], Q[j][c], v);
      Xo[r + (int64_t)(a + i) * ldo] = v;
    }
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
  ++L.syncs;
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

static int syevd_f64(DenseLayer& L, bool vectors, int n, double* A, int lda) {
  SOL_OK(cusolverDnDsyevd(L.sol, vectors ? CUSOLVER_EIG_MODE_VECTOR : CUSOLVER_EIG_MODE_NOVECTOR,
                          CUBLAS_FILL_MODE_LOWER, n, A, lda, L.ev, L.work, L.lwork, L.info));
  return LOBPCG_OK;
}

// Eigenvalues ascending into L.ev, eigenvectors into A (column-major, lda =
// n), by cuSOLVER's FP64 syevd (eig_mode 0) or the FP32 decomposition + FP64
// refinement above (eig_mode 1; FP64 syevd when the FP32 stage fails, meets
// a non-finite value, a cluster wider than kMaxRun or fails the residual
// check).
static int syevd(DenseLayer& L, bool vectors, int n, double* A, int lda) {
  if (L.eig_mode != 1 || n < 2 || lda != n) return syevd_f64(L, vectors, n, A, lda);
  const int64_t nn = (int64_t)n * n;
  const double one = 1.0, zero = 0.0;
  ++L.eig_calls;
  symmetrize_kernel<<<blocks_for(nn), 256, 0, L.st>>>(n, A, lda);
  LAUNCH_OK(L);
  to_f32_kernel<<<blocks_for(nn), 256, 0, L.st>>>(nn, A, L.Af);
  LAUNCH_OK(L);
  SOL_OK(cusolverDnSsyevd(L.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, L.Af, n,
                          L.wf, L.swork, L.lswork, L.info));
  double* X = L.R[0];
  double* X1 = L.R[1];
  double* AX = L.R[2];
  double* S = L.R[3];
  double* G = L.R[4];
  double* E = L.R[5];
  to_f64_kernel<<<blocks_for(nn), 256, 0, L.st>>>(nn, L.Af, X);
  LAUNCH_OK(L);
  const int nb = (int)std::min<int64_t>(kRefBlocks, ceil_div(nn, 256));
  // refinement steps until delta stops shrinking (it levels off at the width
  // of the true clusters) or reaches rounding level; delta and ||A||_F come
  // back to the host after every step
  double delta = INFINITY, normA = 0.0;
  for (int step = 0; step < kMaxRefineSteps; ++step) {
    BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, A, lda, X, n, &zero, AX,
                        n));
    BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n, &one, X, n, AX, n, &zero, S,
                        n));
    BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n, &one, X, n, X, n, &zero, G,
                        n));
    oa_norms_kernel<<<nb, 256, 0, L.st>>>(n, S, G, A, lda, L.part);
    LAUNCH_OK(L);
    oa_update_kernel<<<(unsigned)std::min<int64_t>(4 * 152, ceil_div(nn, 256)), 256, 0, L.st>>>(
        n, S, G, L.part, nb, E, L.scal + 8);
    LAUNCH_OK(L);
    LOB_CUDA_OK(cudaMemcpyAsync(X1, X, nn * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
    BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, X, n, E, n, &one, X1,
                        n));
    std::swap(X, X1);
    LOB_CUDA_OK(cudaMemcpyAsync(L.host, L.scal + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                L.st));
    LOB_CUDA_OK(cudaStreamSynchronize(L.st));
    ++L.syncs;
    const double dnew = L.host[0];
    normA = L.host[1];
    if (!std::isfinite(dnew)) {
      ++L.eig_fallbacks;
      return syevd_f64(L, vectors, n, A, lda);
    }
    const bool level = step > 0 && dnew > 0.25 * delta;
    delta = dnew;
    if (level || delta <= 64.0 * n * kEps * normA) break;
  }
  // the steps leave X^T X - I near 1e-13; one Newton-Schulz step restores
  // orthonormality to rounding level
  BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n, &one, X, n, X, n, &zero, G, n));
  newton_schulz_kernel<<<blocks_for(nn), 256, 0, L.st>>>(n, G);
  LAUNCH_OK(L);
  BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, X, n, G, n, &zero, X1, n));
  std::swap(X, X1);
  BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, A, lda, X, n, &zero, AX,
                      n));
  BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n, &one, X, n, AX, n, &zero, S, n));
  diag_extract_kernel<<<blocks_for(n + 1), 256, 0, L.st>>>(n, S, L.scal + 8, L.ev);
  LAUNCH_OK(L);
  LOB_CUDA_OK(cudaMemcpyAsync(L.host, L.ev, (n + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                              L.st));
  LOB_CUDA_OK(cudaMemcpyAsync(L.host + n + 1, L.info, sizeof(int), cudaMemcpyDeviceToHost, L.st));
  LOB_CUDA_OK(cudaStreamSynchronize(L.st));
  ++L.syncs;
  int info;
  memcpy(&info, L.host + n + 1, sizeof(int));
  const double* d = L.host;
  bool ok = info == 0 && std::isfinite(delta);
  for (int i = 0; ok && i < n; ++i) ok = std::isfinite(d[i]);
  int* perm = L.hint;
  int* runs = L.hint + n;
  int nruns = 0;
  if (ok) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::sort(perm, perm + n, [&](int a, int b) { return d[a] < d[b] || (d[a] == d[b] && a < b); });
    for (int k = 0; k < n && ok;) {
      int e = k + 1;
      while (e < n && d[perm[e]] - d[perm[e - 1]] <= delta) ++e;
      if (e - k > kMaxRun) ok = false;
      if (e - k >= 2) {
        runs[2 * nruns] = k;
        runs[2 * nruns + 1] = e - k;
        ++nruns;
      }
      k = e;
    }
  }
  if (!ok) {
    ++L.eig_fallbacks;
    return syevd_f64(L, vectors, n, A, lda);
  }
  // verification: the coupling of each column to the columns outside its run,
  // sqrt(sum_j s_ij^2), bounds its final residual ||A z - w z||; above
  // 8 sqrt(n) eps ||A||_F the refinement has not converged: FP64 syevd instead
  int* runid = L.hint + n + 2 * nruns;
  for (int k = 0; k < n; ++k) runid[perm[k]] = k;
  for (int r = 0; r < nruns; ++r)
    for (int k = runs[2 * r]; k < runs[2 * r] + runs[2 * r + 1]; ++k) runid[perm[k]] = runs[2 * r];
  const int nint = 2 * n + 2 * nruns;
  LOB_CUDA_OK(cudaMemcpyAsync(L.dint, L.hint, (size_t)nint * sizeof(int), cudaMemcpyHostToDevice,
                              L.st));
  LOB_CUDA_OK(cudaMemsetAsync(L.scal + 10, 0, sizeof(double), L.st));
  offrun_check_kernel<<<blocks_for(n), 256, 0, L.st>>>(n, S, L.dint + n + 2 * nruns,
                                                       (unsigned long long*)(L.scal + 10));
  LAUNCH_OK(L);
  double worst = 0.0;
  LOB_CUDA_OK(cudaMemcpyAsync(L.host, L.scal + 10, sizeof(double), cudaMemcpyDeviceToHost, L.st));
  LOB_CUDA_OK(cudaStreamSynchronize(L.st));
  ++L.syncs;
  worst = L.host[0];
  if (!(worst <= 8.0 * std::sqrt((double)n) * kEps * normA)) {
    ++L.eig_fallbacks;
    return syevd_f64(L, vectors, n, A, lda);
  }
  permute_cols_kernel<<<blocks_for(nn), 256, 0, L.st>>>(n, X, S, L.dint, A, lda, L.ev);
  LAUNCH_OK(L);
  if (nruns > 0) {
    cluster_jacobi_kernel<<<nruns, 256, 0, L.st>>>(n, S, L.dint, L.dint + n, A, lda, L.ev);
    LAUNCH_OK(L);
  }
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
  if (cudaMalloc(&ev, (nmax + 8) * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&d, nmax * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&tau, nmax * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&scal, 16 * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&info, 4 * sizeof(int)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMallocHost(&host, (nmax + 64) * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  for (auto& r : R)
    if (cudaMalloc(&r, mat) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&Af, (size_t)nmax * nmax * sizeof(float)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&wf, nmax * sizeof(float)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&part, 3 * kRefBlocks * sizeof(double)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMalloc(&dint, 4 * nmax * sizeof(int)) != cudaSuccess) return LOBPCG_ERR_OOM;
  if (cudaMallocHost(&hint, 4 * nmax * sizeof(int)) != cudaSuccess) return LOBPCG_ERR_OOM;
  {
    int lws = 0;
    SOL_OK(cusolverDnSsyevd_bufferSize(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                       (int)nmax, Af, (int)nmax, wf, &lws));
    lswork = std::max(lws, 1);
    if (cudaMalloc(&swork, (size_t)lswork * sizeof(float)) != cudaSuccess) return LOBPCG_ERR_OOM;
  }
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
  return dev.init(std::min<int64_t>(nmax, kDevDenseMax));
}

void DenseLayer::release() {
  dev.release();
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
  for (auto& r : R) {
    if (r) cudaFree(r);
    r = nullptr;
  }
  if (Af) cudaFree(Af);
  if (wf) cudaFree(wf);
  if (swork) cudaFree(swork);
  if (part) cudaFree(part);
  if (dint) cudaFree(dint);
  if (hint) cudaFreeHost(hint);
  Af = wf = swork = nullptr;
  part = nullptr;
  dint = hint = nullptr;
  info = nullptr;
  if (sol) cusolverDnDestroy(sol);
  if (blas) cublasDestroy(blas);
  sol = nullptr;
  blas = nullptr;
  nmax = 0;
}

int rr_initial(DenseLayer& L, const double* GA, const double* GB, int nx, double* C,
               double* theta, bool* breakdown) {
  if (dev_rr_fits(L, nx, nx, nx)) return rr_initial_dev(L, GA, GB, nx, C, theta, breakdown);
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
  ++L.syncs;
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

int rr_modified(DenseLayer& L, const double* SAS, const double* SBS, int ns, int nx, int np,
                int nc, bool use_ortho, double tau_skip, bool* flip, double* condR, double* C,
                int* npn_out, double* theta, double* PAP, bool structured) {
  // the explicit pencil (nothing from the identities): the device path
  // factors the X, P block first, then the Schur complement of the W block
  if (!structured && !use_ortho && dev_explicit_fits(L, ns, nx, np))
    return rr_explicit_dev(L, SAS, SBS, ns, nx, np, nc, tau_skip, flip, condR, C, npn_out, theta,
                           PAP);
  // the device path with o = 0 treats S^T B S as one dense block
  const int o = structured ? nx + np : 0;
  if (dev_rr_fits(L, ns, nx, use_ortho ? 0 : ns - o))
    return rr_modified_dev(L, SAS, SBS, ns, nx, o - nx, nc, use_ortho, tau_skip, flip, condR, C,
                           npn_out, theta, PAP);
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
    ++L.syncs;
    int info;
    memcpy(&info, L.host + 1, sizeof(int));
    if (info != 0) {
      *flip = true;
      *condR = INFINITY;
      return LOBPCG_OK;
    }
    // Rinv = R^-1 (one triangular solve with the identity), then cond(R) from
    // power iterations on M = R^T R (still in Tz) and on Rinv Rinv^T
    set_identity_kernel<<<blocks_for((int64_t)ns * ns), 256, 0, L.st>>>(ns, Q2, ld);
    LAUNCH_OK(L);
    BLAS_OK(cublasDtrsm(L.blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                        CUBLAS_DIAG_NON_UNIT, ns, ns, &one, Rm, ld, Q2, ld));
    {
      const size_t bytes = 3 * (size_t)ns * sizeof(float);
      static bool configured[64] = {false};  // the attribute is per device
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev < 0 || dev >= 64 || !configured[dev]) {
        LOB_CUDA_OK(cudaFuncSetAttribute(cond_estimate_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        if (dev >= 0 && dev < 64) configured[dev] = true;
      }
      if (bytes > 200 * 1024) return LOBPCG_ERR_ARG;
      cond_estimate_kernel<<<1, kCondThreads, bytes, L.st>>>(ns, Tz, ld, Q2, ld, L.scal);
      LAUNCH_OK(L);
    }
    double cr;
    if ((rc = to_host(L, &cr, L.scal, sizeof(double)))) return rc;
    *condR = cr;
    if (!(pow(*condR, -3.0) >= tau_skip)) {
      *flip = true;
      return LOBPCG_OK;
    }
    // H <- Rinv^T H Rinv (two GEMMs through M), eig, T Z = D Rinv Z (one
    // GEMM): three DGEMMs (75 us each at n_s = 213) instead of three
    // triangular solves (0.4 ms each).  The products carry errors up to
    // ~cond(R) eps, cond(R) <= ~3.6e4 on this branch; solves to backward
    // error 1e-11 converge with them in the tests
    BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_N, CUBLAS_OP_N, ns, ns, ns, &one, H, ld, Q2, ld, &zero,
                        M, ld));
    BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_T, CUBLAS_OP_N, ns, ns, ns, &one, Q2, ld, M, ld, &zero,
                        H, ld));
    if ((rc = syevd(L, true, ns, H, ld))) return rc;
    BLAS_OK(cublasDgemm(L.blas, CUBLAS_OP_N, CUBLAS_OP_N, ns, ns, ns, &one, Q2, ld, H, ld, &zero,
                        Tz, ld));
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

// C = alpha op(A) op(B) + beta C (column-major): this library's kernels for
// the sizes its device path takes, cuBLAS above them
static int small_gemm(DenseLayer& L, bool ta, bool tb, int m, int n, int k, double alpha,
                      const double* A, int lda, const double* B, int ldb, double beta, double* C,
                      int ldc) {
  if (m <= 0 || n <= 0) return LOBPCG_OK;
  if (L.eig_mode == 0 && m <= L.dev.nmax && n <= 2 * L.dev.nmax)
    return dev_gemm(L, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, nullptr);
  BLAS_OK(cublasDgemm(L.blas, ta ? CUBLAS_OP_T : CUBLAS_OP_N, tb ? CUBLAS_OP_T : CUBLAS_OP_N, m,
                      n, k, &alpha, A, lda, B, ldb, &beta, C, ldc));
  return LOBPCG_OK;
}

int rr_hl(DenseLayer& L, const double* SAS, int ns, int nx, int nc, double* C, int* npn_out,
          double* theta, double* PAP) {
  double* Z = L.A[3];
  double* Y = L.A[4];
  double* T1 = L.A[5];
  double* Tq = L.A[2];
  int rc;
  // eigenpairs of S^T A S into Z, L.ev
  if (dev_rr_fits(L, ns, 0, 0)) {
    int* est = L.dev.ints + 2;
    ++L.dev_calls;
    if ((rc = dev_syev(L, ns, SAS, ns, Z, ns, L.ev, est))) return rc;
    int fl = 0;
    if ((rc = to_host(L, L.host, est, sizeof(int)))) return rc;
    memcpy(&fl, L.host, sizeof(int));
    if (fl != 0) {
      if ((rc = copy_mat(L, ns, ns, SAS, ns, Z, ns))) return rc;
      if ((rc = syevd_fallback(L, ns, Z, ns))) return rc;
    }
  } else {
    if ((rc = copy_mat(L, ns, ns, SAS, ns, Z, ns))) return rc;
    if ((rc = syevd(L, true, ns, Z, ns))) return rc;
  }
  if ((rc = copy_mat(L, ns, nx, Z, ns, C, ns))) return rc;  // C_x = Z_x
  // Theta now: the svqb below reuses the eigenvalue buffer
  LOB_CUDA_OK(cudaMemcpyAsync(theta, L.ev, nx * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
  const int nu = nx - nc;
  int keep = 0;
  if (nu > 0 && ns > nx) {
    // Y = [0; Z_2(:, nc:nx)] - Z_x (Z_x^T [0; Z_2(:, nc:nx)])
    set_zero_kernel<<<blocks_for((int64_t)ns * nu), 256, 0, L.st>>>(ns, nu, Y, ns);
    LAUNCH_OK(L);
    if ((rc = copy_mat(L, ns - nx, nu, Z + nx + (int64_t)nc * ns, ns, Y + nx, ns))) return rc;
    if ((rc = small_gemm(L, true, false, nx, nu, ns - nx, 1.0, Z + nx, ns, Z + nx + (int64_t)nc * ns,
                         ns, 0.0, T1, nx)))
      return rc;
    if ((rc = small_gemm(L, false, false, ns, nu, nx, -1.0, Z, ns, T1, nx, 1.0, Y, ns))) return rc;
    // svqb (Algorithm 4, Euclidean metric): G = Y^T Y, T = D Z_G Theta^-1/2, C_p = Y T
    if ((rc = small_gemm(L, true, false, nu, nu, ns, 1.0, Y, ns, Y, ns, 0.0, T1, nu))) return rc;
    if ((rc = svqb_transform(L, T1, nu, false, nu * kEps, Tq, &keep))) return rc;
    if (keep > 0) {
      if ((rc = small_gemm(L, false, false, ns, keep, nu, 1.0, Y, ns, Tq, nu, 0.0,
                           C + (int64_t)nx * ns, ns)))
        return rc;
      // P^T A P = C_p^T (S^T A S) C_p
      if ((rc = small_gemm(L, false, false, ns, keep, ns, 1.0, SAS, ns, C + (int64_t)nx * ns, ns,
                           0.0, Y, ns)))
        return rc;
      if ((rc = small_gemm(L, true, false, keep, keep, ns, 1.0, C + (int64_t)nx * ns, ns, Y, ns,
                           0.0, PAP, keep)))
        return rc;
    }
  }
  *npn_out = keep;
  return LOBPCG_OK;
}

int svqb_transform(DenseLayer& L, const double* G, int nu, bool drop, double tau, double* T,
                   int* nkeep) {
  *nkeep = 0;
  if (nu <= 0) return LOBPCG_OK;
  if (dev_rr_fits(L, nu, 0, 0)) return svqb_transform_dev(L, G, nu, drop, tau, T, nkeep);
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
             double* SBS, int c0) {
  const int ns = nx + np + nw;
  if (c0 < 0) c0 = nx + np;
  assemble_kernel<<<blocks_for((int64_t)ns * ns), 256, 0, L.st>>>(nx, np, nw, c0, theta, PAP,
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

// Kernel-level entry point of the projected eigensolver (see lobpcg.h).
LOBPCG_EXPORT int lobpcg_syev(int64_t n, double* A, int64_t lda, double* w, int mode,
                              void* stream) {
  if (n <= 0 || n > 8192 || lda < n || !A || !w || mode < 0 || mode > 3 ||
      (mode >= 2 && n > lob::kDevDenseMax))
    return LOBPCG_ERR_ARG;
  lob::DenseLayer L;
  int rc = L.init((cudaStream_t)stream, n);
  bool unchecked = false;
  if (!rc && mode >= 2) {
    // the device-resident eigensolver, cuSOLVER FP64 when its check fails
    double* M = L.A[0];
    double* Z = L.A[1];
    int* status = L.dev.ints + 2;
    rc = lob::copy_mat(L, (int)n, (int)n, A, (int)lda, M, (int)n);
    if (!rc) rc = lob::dev_syev(L, (int)n, M, (int)n, Z, (int)n, L.ev, status);
    int st = 0;
    if (!rc && (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, L.st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(L.st) != cudaSuccess))
      rc = LOBPCG_ERR_CUDA;
    if (!rc && st != 0 && mode == 2) {
      rc = lob::copy_mat(L, (int)n, (int)n, M, (int)n, Z, (int)n);
      if (!rc) rc = lob::syevd_fallback(L, (int)n, Z, (int)n);
    }
    unchecked = !rc && st != 0 && mode == 3;
    if (!rc) rc = lob::copy_mat(L, (int)n, (int)n, Z, (int)n, A, (int)lda);
    if (!rc && cudaMemcpyAsync(w, L.ev, n * sizeof(double), cudaMemcpyDeviceToDevice, L.st) !=
                   cudaSuccess)
      rc = LOBPCG_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(L.st) != cudaSuccess) rc = LOBPCG_ERR_CUDA;
    L.release();
    return unchecked ? LOBPCG_ERR_NOT_CONVERGED : rc;
  }
  if (!rc) {
    L.eig_mode = mode;
    double* M = L.A[0];
    rc = lob::copy_mat(L, (int)n, (int)n, A, (int)lda, M, (int)n);
    if (!rc) rc = lob::syevd(L, true, (int)n, M, (int)n);
    if (!rc) rc = lob::copy_mat(L, (int)n, (int)n, M, (int)n, A, (int)lda);
    if (!rc && cudaMemcpyAsync(w, L.ev, n * sizeof(double), cudaMemcpyDeviceToDevice, L.st) !=
                   cudaSuccess)
      rc = LOBPCG_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(L.st) != cudaSuccess) rc = LOBPCG_ERR_CUDA;
  }
  L.release();
  return rc;
}
