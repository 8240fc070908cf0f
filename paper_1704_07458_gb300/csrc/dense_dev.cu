// Device-resident small dense layer for projected pencils of order n_s <= 256:
// the eigensolver, Cholesky factorisations, triangular inverses, the Householder
// QR of the C_p construction and the small GEMMs of Algorithms 2, 4, 6 and 7,
// all in this library's kernels (no cuSOLVER, no cuBLAS).
//
// GB300's FP64 units run at 1/64 of the FP32 rate (about 2 FP64 FMA per clock
// per SM), so an O(n^3) FP64 step on one SM costs milliseconds at n = 213.
// The layer is therefore built as:
//   * O(n^3) work that must be exact to FP64 (the Ogita-Aishima refinement of
//     the eigenvectors, the products forming the projected matrix and the
//     back-transformation) runs as small FP64 GEMMs spread over the whole GPU
//     (16 x 16 output tiles, a deterministic split of the contraction);
//   * the O(n^3) work that only has to be close (the first eigendecomposition
//     and the Householder QR of C_p) runs in FP32 on one CTA, then FP64
//     refinement steps (eigenvectors) or Newton-Schulz steps (QR factor)
//     restore FP64 accuracy;
//   * the only O(n^3) FP64 factorisation left is the Cholesky factor of the
//     W-block Schur complement (order n_w <= n_x), on one CTA.
// Decisions stay on the device: refinement convergence, clustering and the
// residual check write flags that the host reads once per Rayleigh-Ritz call.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "dense.cuh"

namespace lob {

namespace {

constexpr double kEps64 = 2.220446049250313e-16;  // 2^-52
constexpr int kGT = 16;                            // GEMM output tile
constexpr int kGK = 32;                            // GEMM contraction chunk
constexpr int kMaxKs = 8;                          // GEMM contraction splits
constexpr int kRefSteps = 4;                       // Ogita-Aishima steps
constexpr int kMaxRunDev = 32;                     // cluster width of the final Jacobi

#define DLAUNCH(L)                                                    \
  do {                                                                \
    ++(L).launches;                                                   \
    ++g_launches;                                                     \
    if (cudaPeekAtLastError() != cudaSuccess) return LOBPCG_ERR_CUDA; \
  } while (0)

// ------------------------------------------------------------------ GEMM
// C = alpha op(A) op(B) + beta Cin (column-major; Cin may equal C but neither
// may alias A or B).  One 16 x 16 output tile per CTA (one output per thread)
// and a split of the contraction into ks slices; with ks > 1 every slice
// stores its partial tile, and the CTA that arrives last at the tile's counter
// adds the partials in slice order (deterministic) and resets the counter.
// skip != nullptr: the whole launch is a no-op when *skip is non-zero.
__global__ void __launch_bounds__(256) gemm64_kernel(int m, int n, int k, int ta, int tb,
                                                     double alpha, const double* __restrict__ A,
                                                     int lda, const double* __restrict__ B, int ldb,
                                                     double beta, const double* Cin, int ldcin,
                                                     double* C, int ldc, int ks, int kper,
                                                     double* part, unsigned* cnt, const int* skip) {
  if (skip && *skip) return;
  __shared__ double As[kGK][kGT + 1], Bs[kGK][kGT + 1];
  __shared__ int s_last;
  const int tiles_m = (m + kGT - 1) / kGT;
  const int tile = blockIdx.x, slice = blockIdx.y;
  const int row0 = (tile % tiles_m) * kGT, col0 = (tile / tiles_m) * kGT;
  const int k0 = slice * kper, k1 = min(k, k0 + kper);
  const int t = threadIdx.x, i = t % kGT, j = t / kGT;
  double acc = 0.0;
  for (int kc = k0; kc < k1; kc += kGK) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int e = t + 256 * r;
      int ii, kk;
      if (!ta) { ii = e % kGT; kk = e / kGT; } else { kk = e % kGK; ii = e / kGK; }
      const int row = row0 + ii, kq = kc + kk;
      double a = 0.0;
      if (row < m && kq < k1) a = ta ? A[kq + (int64_t)row * lda] : A[row + (int64_t)kq * lda];
      As[kk][ii] = a;
      int jj;
      if (!tb) { kk = e % kGK; jj = e / kGK; } else { jj = e % kGT; kk = e / kGT; }
      const int col = col0 + jj, kb = kc + kk;
      double b = 0.0;
      if (col < n && kb < k1) b = tb ? B[col + (int64_t)kb * ldb] : B[kb + (int64_t)col * ldb];
      Bs[kk][jj] = b;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGK; ++kk) acc = fma(As[kk][i], Bs[kk][j], acc);
    __syncthreads();
  }
  const int row = row0 + i, col = col0 + j;
  if (ks == 1) {
    if (row < m && col < n) {
      double v = alpha * acc;
      if (beta != 0.0) v = fma(beta, Cin[row + (int64_t)col * ldcin], v);
      C[row + (int64_t)col * ldc] = v;
    }
    return;
  }
  part[((int64_t)tile * ks + slice) * 256 + t] = acc;
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = (atomicAdd(&cnt[tile], 1u) == (unsigned)(ks - 1));
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double sum = 0.0;
  for (int s = 0; s < ks; ++s) sum += __ldcg(&part[((int64_t)tile * ks + s) * 256 + t]);
  if (row < m && col < n) {
    double v = alpha * sum;
    if (beta != 0.0) v = fma(beta, Cin[row + (int64_t)col * ldcin], v);
    C[row + (int64_t)col * ldc] = v;
  }
  if (t == 0) cnt[tile] = 0u;
}

// ------------------------------------------------------- FP64 Cholesky
// A = R^T R in place (upper triangle of A becomes R; the strict lower
// triangle is zeroed), n <= kCholMax, one CTA with A staged in shared memory.
// info[0] = j + 1 for the first non-positive (or non-finite) pivot j, else 0.
constexpr int kCholMax = 160;

__global__ void __launch_bounds__(256) chol64_kernel(int n, double* A, int lda, int* info) {
  extern __shared__ double sa[];  // n x n, column-major, leading dimension n
  __shared__ int s_fail;
  __shared__ double s_r, s_inv;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = (int)blockDim.x >> 5;
  for (int c = warp; c < n; c += nw)
    for (int r = lane; r < n; r += 32) sa[r + c * n] = r <= c ? A[r + (int64_t)c * lda] : 0.0;
  if (t == 0) s_fail = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (t == 0) {  // one square root and one division per step
      const double piv = sa[j + j * n];
      if (!(piv > 0.0) || !isfinite(piv)) {
        s_fail = j + 1;
      } else {
        s_r = sqrt(piv);
        s_inv = 1.0 / s_r;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const double rjj = s_r, inv = s_inv;
    // row j of R: r_jk = a_jk / r_jj (k >= j)
    for (int c = j + t; c < n; c += blockDim.x) sa[j + c * n] = c == j ? rjj : sa[j + c * n] * inv;
    __syncthreads();
    // trailing update of the upper triangle: a_ic -= r_ji r_jc, j < i <= c
    // (a warp per column c, lanes over rows i)
    for (int c = j + 1 + warp; c < n; c += nw) {
      const double rjc = sa[j + c * n];
      for (int i = j + 1 + lane; i <= c; i += 32) sa[i + c * n] = fma(-sa[j + i * n], rjc, sa[i + c * n]);
    }
    __syncthreads();
  }
  __syncthreads();
  for (int c = warp; c < n; c += nw)
    for (int r = lane; r < n; r += 32) A[r + (int64_t)c * lda] = r <= c ? sa[r + c * n] : 0.0;
  if (t == 0) info[0] = s_fail;
}

// X = R^-1 for an upper triangular R (n <= kCholMax), rows from the bottom:
// X(i, i) = 1 / r_ii, X(i, j) = -(sum_{k=i+1..j} r_ik X(k, j)) / r_ii; row i
// of X replaces row i of R in shared memory once all of it is computed.
// skip: no-op when *skip != 0 (the factorisation failed).
__global__ void __launch_bounds__(256) trinv64_kernel(int n, const double* R, int ldr, double* X,
                                                      int ldx, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ double sm[];  // n x n: R, rows turning into X from the bottom
  __shared__ double dinv[kCholMax];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwp = (int)blockDim.x >> 5;
  for (int c = warp; c < n; c += nwp)
    for (int i = lane; i < n; i += 32) sm[i + c * n] = i <= c ? R[i + (int64_t)c * ldr] : 0.0;
  for (int i = t; i < n; i += blockDim.x) dinv[i] = 1.0 / R[i + (int64_t)i * ldr];
  __syncthreads();
  // eight lanes per column c share its dot product (a shuffle reduction), so
  // a row costs (n - i) / 8 dependent steps instead of n - i
  const int sub = t & 7, grp = t >> 3, ngrp = (int)blockDim.x >> 3;
  for (int i = n - 1; i >= 0; --i) {
    const double inv = dinv[i];
    double val[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int h = 0; h < 5; ++h) {
      const int c = i + grp + h * ngrp;  // uniform within each group of 8 lanes
      double sacc = 0.0;
      if (c < n && c > i)
        for (int kk = i + 1 + sub; kk <= c; kk += 8) sacc = fma(sm[i + kk * n], sm[kk + c * n], sacc);
      for (int o = 4; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
      val[h] = c == i ? inv : -sacc * inv;
    }
    __syncthreads();
    if (sub == 0)
      for (int h = 0; h < 5; ++h) {
        const int c = i + grp + h * ngrp;
        if (c < n) sm[i + c * n] = val[h];
      }
    __syncthreads();
  }
  for (int c = warp; c < n; c += nwp)
    for (int i = lane; i < n; i += 32) X[i + (int64_t)c * ldx] = sm[i + c * n];
}

// ------------------------------------------- FP32 tridiagonalisation
// Householder reduction of the symmetric A (FP64, both triangles averaged)
// to tridiagonal T = Q^T A Q in FP32 (the reduction of LAPACK's sytd2, lower
// variant): one CTA, the lower triangle packed in shared memory.  Outputs d
// (n), e (n - 1), the reflectors v_k (column k of V, rows k + 1 .. n - 1,
// v_k[k + 1] = 1), tau (n) and scal[0] = ||A||_F.
__device__ __forceinline__ int pk(int n, int i, int j) {  // (i >= j) packed lower, column-major
  return j * n - (j * (j - 1)) / 2 + (i - j);
}

__global__ void __launch_bounds__(1024, 1) tridiag32_kernel(int n, const double* A, int lda,
                                                            float* d, float* e, float* V, int ldv,
                                                            float* tau, double* scal) {
  extern __shared__ float P[];  // n (n + 1) / 2
  __shared__ float v[256], p[256];
  __shared__ float wpart[32];
  __shared__ float s_tau;
  __shared__ double fro[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double f = 0.0;
  for (int j = warp; j < n; j += 32)
    for (int i = j + lane; i < n; i += 32) {
      const double a = 0.5 * (A[i + (int64_t)j * lda] + A[j + (int64_t)i * lda]);
      P[pk(n, i, j)] = (float)a;
      f += (i == j ? 1.0 : 2.0) * a * a;
    }
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (lane == 0) fro[warp] = f;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < 32; ++w) s += fro[w];
    scal[0] = sqrt(s);
  }
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of the reflected column x = A(k+1 .. n-1, k)
    if (warp == 0) {
      float ss = 0.f;
      for (int i = 1 + lane; i < m; i += 32) {
        const float x = P[pk(n, k + 1 + i, k)];
        ss = fmaf(x, x, ss);
      }
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const float alpha = P[pk(n, k + 1, k)];
      float tk = 0.f, beta = alpha, scale = 0.f;
      if (ss > 0.f) {
        beta = -copysignf(sqrtf(alpha * alpha + ss), alpha);
        tk = (beta - alpha) / beta;
        scale = 1.f / (alpha - beta);
      }
      for (int i = lane; i < m; i += 32) {
        const float vi = i == 0 ? 1.f : (tk != 0.f ? P[pk(n, k + 1 + i, k)] * scale : 0.f);
        v[i] = vi;
        V[(k + 1 + i) + (int64_t)k * ldv] = vi;
      }
      if (lane == 0) {
        s_tau = tk;
        d[k] = P[pk(n, k, k)];
        e[k] = beta;
        tau[k] = tk;
      }
    }
    __syncthreads();
    const float tk = s_tau;
    if (tk == 0.f) continue;  // column already reduced; no barrier needed below
    // p = tau A22 v (warp per row) and the warp partials of p^T v
    float pv = 0.f;
    for (int i = warp; i < m; i += 32) {
      float s = 0.f;
      const int gi = k + 1 + i;
      for (int j = lane; j < m; j += 32) {
        const int gj = k + 1 + j;
        const float a = gi >= gj ? P[pk(n, gi, gj)] : P[pk(n, gj, gi)];
        s = fmaf(a, v[j], s);
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      s *= tk;
      if (lane == 0) p[i] = s;
      pv = fmaf(s, v[i], pv);
    }
    if (lane == 0) wpart[warp] = pv;
    __syncthreads();
    float ptv = 0.f;
    for (int w = 0; w < 32; ++w) ptv += wpart[w];
    const float K = 0.5f * tk * ptv;
    // rank-2 update A22 -= v w^T + w v^T with w = p - K v (lower part)
    for (int j = warp; j < m; j += 32) {
      const float vj = v[j], wj = p[j] - K * v[j];
      for (int i = j + lane; i < m; i += 32) {
        const float vi = v[i], wi = p[i] - K * v[i];
        const int idx = pk(n, k + 1 + i, k + 1 + j);
        P[idx] = P[idx] - (vi * wj + wi * vj);
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    if (n >= 2) {
      d[n - 2] = P[pk(n, n - 2, n - 2)];
      d[n - 1] = P[pk(n, n - 1, n - 1)];
      e[n - 2] = P[pk(n, n - 1, n - 2)];
      tau[n - 2] = 0.f;
    } else {
      d[0] = P[0];
    }
    tau[n - 1] = 0.f;
  }
}

// The same reduction with the lower triangle kept in a full n x ld array
// (ld = n rounded up to odd, n <= kTridFull) in shared memory: the product
// p = tau A22 v runs one thread per row (row i reads A(i, j), j <= i, along
// its row and A(j, i), j > i, down its column; with an odd ld both patterns
// are free of bank conflicts across a warp), four accumulators per thread;
// the rank-2 update touches the lower triangle only.
constexpr int kTridFull = 223;

__global__ void __launch_bounds__(1024, 1) tridiag32_full_kernel(int n, const double* A, int lda,
                                                                 float* d, float* e, float* V,
                                                                 int ldv, float* tau,
                                                                 double* scal) {
  extern __shared__ float F[];  // n x ld, F[i * ld + j] = A(i, j) for j <= i
  __shared__ float v[256], p[256];
  __shared__ float wpart[32];
  __shared__ float s_tau;
  __shared__ double fro[32];
  const int ld = n | 1;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double f = 0.0;
  for (int i = warp; i < n; i += 32)
    for (int j = lane; j <= i; j += 32) {
      const double a = 0.5 * (A[i + (int64_t)j * lda] + A[j + (int64_t)i * lda]);
      F[i * ld + j] = (float)a;
      f += (i == j ? 1.0 : 2.0) * a * a;
    }
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (lane == 0) fro[warp] = f;
  __syncthreads();
  if (t == 0) {
    double sacc = 0.0;
    for (int w = 0; w < 32; ++w) sacc += fro[w];
    scal[0] = sqrt(sacc);
  }
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    const int o = k + 1;  // first row / column of the trailing block
    if (warp == 0) {
      // x = A(k+1 .. n-1, k): column k below the diagonal (stride ld)
      float ss = 0.f;
      for (int i = 1 + lane; i < m; i += 32) {
        const float x = F[(o + i) * ld + k];
        ss = fmaf(x, x, ss);
      }
      for (int q = 16; q > 0; q >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, q);
      const float alpha = F[o * ld + k];
      float tk = 0.f, beta = alpha, scale = 0.f;
      if (ss > 0.f) {
        beta = -copysignf(sqrtf(alpha * alpha + ss), alpha);
        tk = (beta - alpha) / beta;
        scale = 1.f / (alpha - beta);
      }
      for (int i = lane; i < m; i += 32) {
        const float vi = i == 0 ? 1.f : (tk != 0.f ? F[(o + i) * ld + k] * scale : 0.f);
        v[i] = vi;
        V[(o + i) + (int64_t)k * ldv] = vi;
      }
      if (lane == 0) {
        s_tau = tk;
        d[k] = F[k * ld + k];
        e[k] = beta;
        tau[k] = tk;
      }
    }
    __syncthreads();
    const float tk = s_tau;
    if (tk == 0.f) continue;
    // p_i = tau sum_j A22(i, j) v_j: four consecutive lanes per row, lane
    // sub of a row takes the j = sub (mod 4) terms of the stored lower
    // triangle (row part j <= i, column part j > i), a shuffle sums them
    float pv = 0.f;
    {
      const int r = t >> 2, sub = t & 3;
      float a0 = 0.f, a1 = 0.f;
      if (r < m) {
        const int gi = o + r;
        const float* row = F + gi * ld + o;  // A(gi, o + j), j <= r
        int j = sub;
        for (; j + 4 <= r; j += 8) {
          a0 = fmaf(row[j], v[j], a0);
          a1 = fmaf(row[j + 4], v[j + 4], a1);
        }
        for (; j <= r; j += 4) a0 = fmaf(row[j], v[j], a0);
        // j > r: A(o + j, gi) = F[(o + j) * ld + gi]; first j = r + 1 + ((sub - r - 1) mod 4)
        j = r + 1 + ((sub - r - 1) & 3);
        for (; j + 4 < m; j += 8) {
          a0 = fmaf(F[(o + j) * ld + gi], v[j], a0);
          a1 = fmaf(F[(o + j + 4) * ld + gi], v[j + 4], a1);
        }
        for (; j < m; j += 4) a0 = fmaf(F[(o + j) * ld + gi], v[j], a0);
      }
      float sacc = a0 + a1;
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 2);
      if (r < m && sub == 0) {
        sacc *= tk;
        p[r] = sacc;
        pv = sacc * v[r];
      }
    }
    for (int q = 16; q > 0; q >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, q);
    if (lane == 0) wpart[warp] = pv;
    __syncthreads();
    float ptv = 0.f;
    for (int w = 0; w < 32; ++w) ptv += wpart[w];
    const float K = 0.5f * tk * ptv;
    // rank-2 update of the lower triangle: A22(i, j) -= v_i w_j + w_i v_j
    for (int i = warp; i < m; i += 32) {
      float* row = F + (o + i) * ld + o;
      const float vi = v[i], wi = p[i] - K * v[i];
      for (int j = lane; j <= i; j += 32) row[j] = row[j] - (vi * (p[j] - K * v[j]) + wi * v[j]);
    }
    __syncthreads();
  }
  if (t == 0) {
    if (n >= 2) {
      d[n - 2] = F[(n - 2) * ld + (n - 2)];
      d[n - 1] = F[(n - 1) * ld + (n - 1)];
      e[n - 2] = F[(n - 1) * ld + (n - 2)];
      tau[n - 2] = 0.f;
    } else {
      d[0] = F[0];
    }
    tau[n - 1] = 0.f;
  }
}

// --------------------------- tridiagonal eigenvalues and eigenvectors
// One thread per eigenvalue index j (32 per CTA): bisection on the Sturm
// count for lambda_j (FP32), then two steps of inverse iteration with T -
// lambda_j I factored by Gaussian elimination with partial pivoting (the
// method of LAPACK's stein), from a start vector hashed from j so that
// members of a tight cluster start in different directions.  Per-thread
// work arrays live in shared memory interleaved by lane.  Y(:, j) (FP32,
// n x n column-major) receives the unit eigenvector of T; lam[j] the
// eigenvalue.
__device__ __forceinline__ float hash_unit(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;  // [-1, 1)
}

// lam[j], j = 0 .. n-1: the eigenvalues of T by multisection on the Sturm
// count (count(x) = number of eigenvalues below x, LAPACK's pivmin guard),
// four lanes per eigenvalue evaluating four interior points of the interval
// at once (each round narrows it five-fold), to FP32 resolution.
__global__ void __launch_bounds__(256) bisect_kernel(int n, const float* __restrict__ dg,
                                                     const float* __restrict__ eg,
                                                     float* __restrict__ lam) {
  __shared__ float d[256], e2[256];
  __shared__ float s_gl, s_gu, s_piv;
  const int t = threadIdx.x;
  for (int i = t; i < n; i += blockDim.x) {
    d[i] = dg[i];
    const float ei = i + 1 < n ? eg[i] : 0.f;
    e2[i] = ei * ei;
  }
  __syncthreads();
  if (t == 0) {
    float gl = FLT_MAX, gu = -FLT_MAX, emax2 = 0.f;
    for (int i = 0; i < n; ++i) {
      const float r = (i > 0 ? sqrtf(e2[i - 1]) : 0.f) + (i + 1 < n ? sqrtf(e2[i]) : 0.f);
      gl = fminf(gl, d[i] - r);
      gu = fmaxf(gu, d[i] + r);
      emax2 = fmaxf(emax2, e2[i]);
    }
    const float tnorm = fmaxf(fabsf(gl), fabsf(gu));
    const float pivmin = FLT_MIN * fmaxf(1.f, emax2);
    s_gl = gl - 2.f * FLT_EPSILON * tnorm * n - pivmin;
    s_gu = gu + 2.f * FLT_EPSILON * tnorm * n + pivmin;
    s_piv = pivmin;
  }
  __syncthreads();
  const int g = (blockIdx.x * blockDim.x + t) >> 2, q = t & 3;
  const bool active = g < n;
  const float pivmin = s_piv;
  float lo = s_gl, hi = s_gu;
  for (int round = 0; round < 24; ++round) {
    const float wdt = hi - lo;
    const bool conv = !(wdt > 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)) + pivmin);
    // the four lanes of a group share lo, hi: they stop together
    const float x = lo + (float)(q + 1) * 0.2f * wdt;
    int c = 0;
    if (active && !conv) {
      float qq = 1.f;
      for (int i = 0; i < n; ++i) {
        qq = d[i] - x - (i > 0 ? e2[i - 1] / qq : 0.f);
        if (fabsf(qq) < pivmin) qq = -pivmin;
        c += qq < 0.f;
      }
    }
    // first of the four points with count > g: the eigenvalue lies below it
    const unsigned above = __ballot_sync(0xffffffffu, active && !conv && c > g);
    const unsigned grp = (above >> ((t & 31) & ~3)) & 0xFu;
    const int first = grp ? __ffs(grp) - 1 : 4;
    const float x0 = lo + (float)first * 0.2f * wdt, x1 = lo + (float)(first + 1) * 0.2f * wdt;
    if (!conv) {
      lo = first == 0 ? lo : x0;
      hi = first == 4 ? hi : x1;
    }
  }
  if (active && q == 0) lam[g] = 0.5f * (lo + hi);
}

// Inverse iteration (two steps) for eigenvalue lam[j] of T, one thread per j
// (32 per CTA), with T - lam_j I factored by Gaussian elimination with
// partial pivoting (the method of LAPACK's stein), from a start vector hashed
// from j so that members of a tight cluster start in different directions.
// Per-thread work arrays live in shared memory interleaved by lane.  Y(:, j)
// (FP32, n x n column-major) receives the unit eigenvector of T.
__global__ void __launch_bounds__(32) tridiag_eig_kernel(int n, const float* __restrict__ dg,
                                                         const float* __restrict__ eg,
                                                         const float* __restrict__ lam,
                                                         float* __restrict__ Y, int ldy) {
  extern __shared__ float ws[];  // d, e, e^2 (3 n) then 6 arrays of n x 32
  float* d = ws;
  float* e = ws + n;
  float* e2 = ws + 2 * n;
  float* u0 = ws + 3 * n;
  float* u1 = u0 + 32 * n;
  float* u2 = u1 + 32 * n;
  float* lm = u2 + 32 * n;
  float* y = lm + 32 * n;
  float* sw = y + 32 * n;  // 1: rows i and i + 1 were swapped at step i
  const int lane = threadIdx.x;
  for (int i = lane; i < n; i += 32) {
    d[i] = dg[i];
    const float ei = i + 1 < n ? eg[i] : 0.f;
    e[i] = ei;
    e2[i] = ei * ei;
  }
  __syncwarp();
  float gl = FLT_MAX, gu = -FLT_MAX, emax2 = 0.f;
  for (int i = 0; i < n; ++i) {
    const float r = (i > 0 ? fabsf(e[i - 1]) : 0.f) + (i + 1 < n ? fabsf(e[i]) : 0.f);
    gl = fminf(gl, d[i] - r);
    gu = fmaxf(gu, d[i] + r);
    emax2 = fmaxf(emax2, e2[i]);
  }
  const float tnorm = fmaxf(fabsf(gl), fabsf(gu));
  const float pivmin = FLT_MIN * fmaxf(1.f, emax2);
  const int j = blockIdx.x * 32 + lane;
  if (j >= n) return;
  const float L = lam[j];
  // ---- LU with partial pivoting of T - L I (rows i, i + 1 may swap):
  // U has diagonal u0, superdiagonals u1, u2; multipliers in lm, swaps in sw
  const float pert = FLT_EPSILON * tnorm + pivmin;
#define AT(arr, i) arr[(i) * 32 + lane]
  float diag = d[0] - L, sup = n > 1 ? e[0] : 0.f;
  for (int i = 0; i + 1 < n; ++i) {
    const float sub = e[i], nd = d[i + 1] - L, ns = i + 2 < n ? e[i + 1] : 0.f;
    if (fabsf(diag) >= fabsf(sub)) {
      if (diag == 0.f) diag = pert;
      const float mlt = sub / diag;
      AT(lm, i) = mlt;
      AT(sw, i) = 0.f;
      AT(u0, i) = diag;
      AT(u1, i) = sup;
      AT(u2, i) = 0.f;
      diag = nd - mlt * sup;
      sup = ns;
    } else {
      const float mlt = diag / sub;
      AT(lm, i) = mlt;
      AT(sw, i) = 1.f;
      AT(u0, i) = sub;
      AT(u1, i) = nd;
      AT(u2, i) = ns;
      diag = sup - mlt * nd;
      sup = -mlt * ns;
    }
  }
  if (fabsf(diag) < pert) diag = diag < 0.f ? -pert : pert;
  AT(u0, n - 1) = diag;
  for (int i = 0; i < n; ++i) AT(y, i) = hash_unit((uint32_t)j, (uint32_t)i);
  for (int step = 0; step < 2; ++step) {
    // forward: apply the row operations
    for (int i = 0; i + 1 < n; ++i) {
      const float c = AT(lm, i);
      if (AT(sw, i) == 0.f) {
        AT(y, i + 1) -= c * AT(y, i);
      } else {
        const float yi = AT(y, i), yi1 = AT(y, i + 1);
        AT(y, i) = yi1;
        AT(y, i + 1) = yi - c * yi1;
      }
    }
    // back substitution with U
    float nrm = 0.f;
    for (int i = n - 1; i >= 0; --i) {
      float s = AT(y, i);
      if (i + 1 < n) s -= AT(u1, i) * AT(y, i + 1);
      if (i + 2 < n) s -= AT(u2, i) * AT(y, i + 2);
      float u = AT(u0, i);
      if (fabsf(u) < pert) u = u < 0.f ? -pert : pert;
      const float xi = s / u;
      AT(y, i) = xi;
      nrm = fmaxf(nrm, fabsf(xi));
    }
    const float sc = nrm > 0.f ? 1.f / nrm : 1.f;
    for (int i = 0; i < n; ++i) AT(y, i) *= sc;
  }
  float s2 = 0.f;
  for (int i = 0; i < n; ++i) s2 = fmaf(AT(y, i), AT(y, i), s2);
  const float inv = s2 > 0.f ? rsqrtf(s2) : 0.f;
  for (int i = 0; i < n; ++i) Y[i + (int64_t)j * ldy] = AT(y, i) * inv;
#undef AT
}

// Tight clusters of the tridiagonal spectrum (consecutive eigenvalues closer
// than 1e-5 ||T||, where inverse iteration in FP32 cannot separate the
// vectors): each cluster's vectors are orthonormalised in eigenvalue order
// by modified Gram-Schmidt (one warp per cluster, clusters found by thread
// 0).  Vectors of well separated eigenvalues are left as they are.
__global__ void __launch_bounds__(1024, 1) cluster_orth_kernel(int n, const float* __restrict__ lam,
                                                               float* __restrict__ Y, int ldy) {
  __shared__ int runs[2 * 128];
  __shared__ int nruns;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) {
    float tn = 0.f;
    for (int i = 0; i < n; ++i) tn = fmaxf(tn, fabsf(lam[i]));
    const float thr = 1e-5f * tn;
    int nr = 0;
    for (int a = 0; a < n;) {
      int b = a + 1;
      while (b < n && lam[b] - lam[b - 1] <= thr) ++b;
      if (b - a >= 2 && nr < 128) {
        runs[2 * nr] = a;
        runs[2 * nr + 1] = b - a;
        ++nr;
      }
      a = b;
    }
    nruns = nr;
  }
  __syncthreads();
  for (int r = warp; r < nruns; r += 32) {
    const int a = runs[2 * r], m = runs[2 * r + 1];
    for (int c = a; c < a + m; ++c) {
      float* yc = Y + (int64_t)c * ldy;
      for (int pass = 0; pass < 2; ++pass)
        for (int b = a; b < c; ++b) {
          const float* yb = Y + (int64_t)b * ldy;
          float s = 0.f;
          for (int i = lane; i < n; i += 32) s = fmaf(yb[i], yc[i], s);
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          for (int i = lane; i < n; i += 32) yc[i] = fmaf(-s, yb[i], yc[i]);
          __syncwarp();
        }
      float s = 0.f;
      for (int i = lane; i < n; i += 32) s = fmaf(yc[i], yc[i], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const float inv = s > 0.f ? rsqrtf(s) : 0.f;
      for (int i = lane; i < n; i += 32) yc[i] *= inv;
      __syncwarp();
    }
  }
}

// Z = Q Y with Q = H_0 H_1 ... H_{n-3}, H_k = I - tau_k v_k v_k^T: reflectors
// applied from the last to the first, each column of Y independently (one
// half-warp per column, 16 columns per CTA).  The reflectors are staged in
// shared memory (packed, strictly lower part) so that the n sequential
// reflector steps read no global memory.  Z is written in FP64.
__device__ __forceinline__ int vpk(int n, int k) {  // start of reflector k (rows k+1 .. n-1)
  return k * (n - 1) - (k * (k - 1)) / 2;
}

__global__ void __launch_bounds__(256) backtransform_kernel(int n, const float* __restrict__ V,
                                                            int ldv, const float* __restrict__ tau,
                                                            const float* __restrict__ Y, int ldy,
                                                            double* __restrict__ Z, int ldz) {
  extern __shared__ float bs[];
  float* vp = bs;                          // n (n - 1) / 2
  float* ys = bs + (n * (n - 1)) / 2;      // 16 x n
  __shared__ float ts[256];
  const int t = threadIdx.x, c = t >> 4, r = t & 15;
  for (int k = 0; k + 1 < n; ++k) {
    const int base = vpk(n, k), len = n - 1 - k;
    for (int i = t; i < len; i += blockDim.x) vp[base + i] = V[(k + 1 + i) + (int64_t)k * ldv];
  }
  for (int k = t; k < n; k += blockDim.x) ts[k] = tau[k];
  const int col = blockIdx.x * 16 + c;
  const bool active = col < n;
  float* y = ys + c * n;
  if (active)
    for (int i = r; i < n; i += 16) y[i] = Y[i + (int64_t)col * ldy];
  __syncthreads();
  const unsigned mask = 0xFFFFu << (16 * ((t >> 4) & 1));
  for (int k = n - 3; k >= 0; --k) {
    const float tk = ts[k];
    if (tk == 0.f) continue;
    const float* v = vp + vpk(n, k) - (k + 1);  // v[i] for i = k+1 .. n-1
    float sacc = 0.f;
    if (active)
      for (int i = k + 1 + r; i < n; i += 16) sacc = fmaf(v[i], y[i], sacc);
    for (int o = 8; o > 0; o >>= 1) sacc += __shfl_xor_sync(mask, sacc, o);
    sacc *= tk;
    if (active)
      for (int i = k + 1 + r; i < n; i += 16) y[i] = fmaf(-sacc, v[i], y[i]);
    __syncwarp(mask);
  }
  if (active)
    for (int i = r; i < n; i += 16) Z[i + (int64_t)col * ldz] = (double)y[i];
}

// -------------------------------------------- FP64 refinement steps
// One Ogita-Aishima step from [G, S] = X^T [X, A X] (n x 2n, column-major):
// d_i = s_ii / g_ii, R = I - G, delta = 2 (||S - diag(d) G||_F + ||A||_F ||R||_F),
// E_ij = (s_ij + d_j r_ij) / (d_j - d_i) when |d_j - d_i| > delta and that
// quotient is below 1e-2 (a first-order correction), else r_ij / 2 (the pair
// is treated as a cluster: orthogonalised only); E_ii = r_ii / 2.  Sets
// done[0] when delta <= 64 n eps ||A||_F (converged: later steps skip).
// Two kernels over the whole GPU: partial norms and d, then delta and E.
constexpr int kOaBlocks = 64;

__global__ void __launch_bounds__(256) oa_norms_kernel(int n, const double* __restrict__ GS,
                                                       double* __restrict__ part,
                                                       double* __restrict__ dvec, const int* done) {
  if (*done) return;
  __shared__ double red[2][8];
  const double* G = GS;
  const double* S = GS + (int64_t)n * n;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double a = 0.0, b = 0.0;
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + t; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    const double g = G[e], sv = S[e];
    if (i == j) {
      const double dd = sv / g;
      dvec[i] = dd;
      a = fma(sv - dd * g, sv - dd * g, a);
      b = fma(1.0 - g, 1.0 - g, b);
    } else {
      a = fma(sv, sv, a);
      b = fma(g, g, b);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    red[0][warp] = a;
    red[1][warp] = b;
  }
  __syncthreads();
  if (t == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < 8; ++w) {
      sa += red[0][w];
      sb += red[1][w];
    }
    part[2 * blockIdx.x] = sa;
    part[2 * blockIdx.x + 1] = sb;
  }
}

__global__ void __launch_bounds__(256) oa_e_kernel(int n, const double* __restrict__ GS,
                                                   const double* __restrict__ part,
                                                   const double* __restrict__ dvec,
                                                   const double* __restrict__ scal,
                                                   double* __restrict__ E, int* done,
                                                   double* delta_out,
                                                   unsigned long long* emax) {
  if (*done) return;
  __shared__ double s_delta;
  __shared__ unsigned long long s_max[8];
  const double* G = GS;
  const double* S = GS + (int64_t)n * n;
  if (threadIdx.x < 32) {  // fixed-order sum of the partials (every CTA alike)
    double sa = 0.0, sb = 0.0;
    for (int q = threadIdx.x; q < kOaBlocks; q += 32) {
      sa += part[2 * q];
      sb += part[2 * q + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if (threadIdx.x == 0) s_delta = 2.0 * (sqrt(sa) + scal[0] * sqrt(sb));
  }
  __syncthreads();
  const double delta = s_delta;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long m = 0;
  if (e < (int64_t)n * n) {
    const int i = (int)(e % n), j = (int)(e / n);
    const double r = (i == j ? 1.0 : 0.0) - G[e];
    double out = 0.5 * r;
    if (i != j) {
      const double di = dvec[i], dj = dvec[j];
      const double gap = dj - di, num = S[e] + dj * r;
      if (fabs(gap) > delta && fabs(num) <= 1e-2 * fabs(gap)) out = num / gap;
    }
    E[e] = out;
    m = (unsigned long long)__double_as_longlong(fabs(out));
  }
  // largest |E_ij| of the step (non-negative doubles order as their bits)
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long mm = 0;
    for (int w = 0; w < 8; ++w) mm = max(mm, s_max[w]);
    atomicMax(emax, mm);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    delta_out[0] = delta;
    // converged: the update of this step and every later step are skipped
    if (!(delta > 64.0 * n * kEps64 * scal[0])) done[0] = 1;
  }
}

// Skip flag of the next refinement step: set when this step was skipped or
// converged (done) or its largest correction |E_ij| was at most 1e-10 (a
// further step would change the vectors below FP64 resolution).  The
// Newton-Schulz steps that follow always run: a first-order step leaves an
// orthogonality defect of order |s_ij - s_ji| / |d_j - d_i| (the rounding
// asymmetry of X^T A X over the gap) even when its corrections are tiny.
__global__ void oa_next_kernel(const int* cur, const unsigned long long* emax, int* next) {
  if (threadIdx.x == 0)
    next[0] = (cur[0] || __longlong_as_double((long long)emax[0]) <= 1e-10) ? 1 : 0;
}

// Final pass on S = X^T A X, G = X^T X of the refined X (one CTA): order by
// d_i = s_ii, and group the sorted positions into runs: positions k < j join
// one run (with everything between them) when |s_ij| > 8 eps ||A||_F, i.e.
// pairs the first-order steps did not decouple (clusters, and pairs whose
// correction the steps' guard refused).  Outside the runs every coupling is
// then below 8 eps ||A||_F (row norms below 8 sqrt(n) eps ||A||_F), so the
// run blocks' FP64 Jacobi finishes the decomposition.  Checks ||I - G||_F at
// rounding level, finite values and runs no wider than kMaxRunDev; writes the
// permutation, the runs, the eigenvalues w (ascending) and status[0] = 0 on
// success, else a bit mask (1 orthogonality, 2 wide run, 8 non-finite) and
// the caller falls back.
__global__ void __launch_bounds__(1024, 1) eig_finalize_kernel(int n, const double* __restrict__ GS,
                                                               const double* __restrict__ scal,
                                                               int* __restrict__ perm,
                                                               int* __restrict__ runs,
                                                               int* __restrict__ nruns_out,
                                                               double* __restrict__ w,
                                                               int* status) {
  __shared__ double dv[256];
  __shared__ int pm[256], pos[256], reach[256];
  __shared__ double red[32];
  __shared__ int s_bad;
  const double* G = GS;
  const double* S = GS + (int64_t)n * n;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t < n) dv[t] = S[t + (int64_t)t * n];
  if (t == 0) s_bad = 0;
  __syncthreads();
  if (t < n) {  // rank of d_t (ties by index)
    int r = 0;
    const double x = dv[t];
    for (int j = 0; j < n; ++j) r += (dv[j] < x || (dv[j] == x && j < t)) ? 1 : 0;
    pm[r] = t;
    pos[t] = r;
    if (!isfinite(x)) atomicOr(&s_bad, 8);
  }
  double b = 0.0;
  for (int e = t; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    const double r = (i == j ? 1.0 : 0.0) - G[e];
    b = fma(r, r, b);
  }
  for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
  if (lane == 0) red[warp] = b;
  __syncthreads();
  const double thr = 8.0 * kEps64 * scal[0];
  // furthest sorted position coupled to each position (a warp per column of
  // S, contiguous reads; S is symmetric to rounding)
  for (int tt = warp; tt < n; tt += 32) {
    const int i = pm[tt];
    int rmax = tt;
    for (int j = lane; j < n; j += 32)
      if (j != i && !(fabs(S[j + (int64_t)i * n]) <= thr)) rmax = max(rmax, pos[j]);
    for (int o = 16; o > 0; o >>= 1) rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if (lane == 0) reach[tt] = rmax;
  }
  __syncthreads();
  if (t == 0) {
    double sb = 0.0;
    for (int q = 0; q < 32; ++q) sb += red[q];
    if (!(sqrt(sb) <= 64.0 * n * kEps64)) s_bad |= 1;
    int nr = 0;
    for (int k = 0; k < n;) {
      int e2 = reach[k];
      for (int j = k; j <= e2; ++j) e2 = max(e2, reach[j]);
      const int m = e2 - k + 1;
      if (m > kMaxRunDev) s_bad |= 2;
      if (m >= 2) {
        runs[2 * nr] = k;
        runs[2 * nr + 1] = m;
        ++nr;
      }
      k = e2 + 1;
    }
    nruns_out[0] = nr;
  }
  __syncthreads();
  if (t < n) {
    perm[t] = pm[t];
    w[t] = dv[pm[t]];
  }
  if (t == 0) status[0] = s_bad;
}

// Zo(:, k) = X(:, perm[k]) (column permutation into the output).
__global__ void permute_cols_dev_kernel(int n, const double* __restrict__ X, int ldxx,
                                        const int* __restrict__ perm, double* __restrict__ Zo,
                                        int ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int r = (int)(e % n), k = (int)(e / n);
  Zo[r + (int64_t)k * ldo] = X[r + (int64_t)perm[k] * ldxx];
}

// Cyclic Jacobi (Golub & Van Loan, Sec. 8.5) on the FP64 block S(perm[a + i],
// perm[a + j]) of each run [a, a + m), one CTA per run (CTAs beyond the run
// count exit), then Zo(:, a : a + m) <- Zo(:, a : a + m) Q and w(a : a + m)
// the block's eigenvalues ascending.
__global__ void __launch_bounds__(256) run_jacobi_kernel(int n, const double* __restrict__ GS,
                                                         const int* __restrict__ perm,
                                                         const int* __restrict__ runs,
                                                         const int* __restrict__ nruns,
                                                         double* __restrict__ Zo, int ldo,
                                                         double* __restrict__ w) {
  if ((int)blockIdx.x >= nruns[0]) return;
  if (runs[2 * blockIdx.x + 1] > kMaxRunDev) return;  // flagged by the finalize pass
  const double* S = GS + (int64_t)n * n;
  __shared__ double M[kMaxRunDev][kMaxRunDev + 1], Q[kMaxRunDev][kMaxRunDev + 1];
  __shared__ double ev[kMaxRunDev];
  __shared__ int order[kMaxRunDev];
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
      for (int pp = 0; pp < m - 1; ++pp)
        for (int qq = pp + 1; qq < m; ++qq) {
          const double apq = M[pp][qq];
          if (apq == 0.0) continue;
          const double tau = (M[qq][qq] - M[pp][pp]) / (2.0 * apq);
          const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
          const double c = 1.0 / sqrt(1.0 + tt * tt), s = tt * c;
          __syncwarp();
          for (int kk = lane; kk < m; kk += 32) {
            const double mkp = M[kk][pp], mkq = M[kk][qq];
            M[kk][pp] = c * mkp - s * mkq;
            M[kk][qq] = s * mkp + c * mkq;
            const double qkp = Q[kk][pp], qkq = Q[kk][qq];
            Q[kk][pp] = c * qkp - s * qkq;
            Q[kk][qq] = s * qkp + c * qkq;
          }
          __syncwarp();
          for (int kk = lane; kk < m; kk += 32) {
            const double mpk = M[pp][kk], mqk = M[qq][kk];
            M[pp][kk] = c * mpk - s * mqk;
            M[qq][kk] = s * mpk + c * mqk;
          }
          __syncwarp();
        }
    }
    if (lane == 0) {
      for (int i = 0; i < m; ++i) {
        ev[i] = M[i][i];
        order[i] = i;
      }
      for (int i = 1; i < m; ++i)
        for (int j = i; j > 0 && ev[order[j]] < ev[order[j - 1]]; --j) {
          const int tmp = order[j];
          order[j] = order[j - 1];
          order[j - 1] = tmp;
        }
    }
  }
  __syncthreads();
  for (int i = tid; i < m; i += blockDim.x) w[a + i] = ev[order[i]];
  for (int r = tid; r < n; r += blockDim.x) {
    double x[kMaxRunDev];
    for (int j = 0; j < m; ++j) x[j] = Zo[r + (int64_t)(a + j) * ldo];
    for (int i = 0; i < m; ++i) {
      const int c = order[i];
      double v = 0.0;
      for (int j = 0; j < m; ++j) v = fma(x[j], Q[j][c], v);
      Zo[r + (int64_t)(a + i) * ldo] = v;
    }
  }
}

// ------------------------------------------ FP32 Householder QR (C_p)
// Thin QR of the tall M (m x c, m > c, column-major FP64): Householder QR in
// FP32 on one CTA (M in shared memory), then Q (m x c) formed by applying
// the reflectors to the first c columns of the identity, written in FP64.
// Each reflector is column-wise backward stable, so the span of a column of
// M is kept to FP32 accuracy relative to that column's own norm whatever
// the other columns' norms; the caller restores FP64 orthonormality.
__global__ void __launch_bounds__(1024, 1) qr32_kernel(int m, int c, const double* __restrict__ M,
                                                       int ldm, double* __restrict__ Q, int ldq) {
  extern __shared__ float qs[];
  float* a = qs;          // m x c
  float* q = qs + m * c;  // m x c
  __shared__ float tv[256];
  __shared__ float s_tau;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int e = t; e < m * c; e += blockDim.x) {
    const int i = e % m, j = e / m;
    a[e] = (float)M[i + (int64_t)j * ldm];
    q[e] = i == j ? 1.f : 0.f;
  }
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    if (warp == 0) {
      float ss = 0.f;
      for (int i = j + 1 + lane; i < m; i += 32) ss = fmaf(a[i + j * m], a[i + j * m], ss);
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const float alpha = a[j + j * m];
      float tk = 0.f, beta = alpha, scale = 0.f;
      if (ss > 0.f) {
        beta = -copysignf(sqrtf(alpha * alpha + ss), alpha);
        tk = (beta - alpha) / beta;
        scale = 1.f / (alpha - beta);
      }
      if (lane == 0) {
        s_tau = tk;
        tv[j] = tk;
      }
      __syncwarp();
      for (int i = j + 1 + lane; i < m; i += 32) a[i + j * m] = tk != 0.f ? a[i + j * m] * scale : 0.f;
      if (lane == 0) a[j + j * m] = beta;
    }
    __syncthreads();
    const float tk = s_tau;
    if (tk != 0.f) {
      // columns j + 1 .. c - 1: x -= tau v (v^T x), v = [1; a(j+1:m, j)]
      for (int cc = j + 1 + warp; cc < c; cc += 32) {
        float s = 0.f;
        for (int i = j + lane; i < m; i += 32)
          s = fmaf(i == j ? 1.f : a[i + j * m], a[i + cc * m], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        s *= tk;
        for (int i = j + lane; i < m; i += 32)
          a[i + cc * m] = fmaf(-s, i == j ? 1.f : a[i + j * m], a[i + cc * m]);
      }
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{c-1} I(:, 0:c): reflectors applied from the last
  for (int j = c - 1; j >= 0; --j) {
    const float tk = tv[j];
    if (tk != 0.f)
      for (int cc = warp; cc < c; cc += 32) {
        float s = 0.f;
        for (int i = j + lane; i < m; i += 32)
          s = fmaf(i == j ? 1.f : a[i + j * m], q[i + cc * m], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        s *= tk;
        for (int i = j + lane; i < m; i += 32)
          q[i + cc * m] = fmaf(-s, i == j ? 1.f : a[i + j * m], q[i + cc * m]);
      }
    __syncthreads();
  }
  for (int e = t; e < m * c; e += blockDim.x) {
    const int i = e % m, j = e / m;
    Q[i + (int64_t)j * ldq] = (double)q[e];
  }
}

// ------------------------------------------------- small helpers
// D = S (rows x cols), skipped when *skip != 0
__global__ void copy_skip_kernel(int rows, int cols, const double* __restrict__ S, int lds,
                                 double* __restrict__ D, int ldd, const int* skip) {
  if (skip && *skip) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  D[i + (int64_t)j * ldd] = S[i + (int64_t)j * lds];
}

// order 1: Z = [1], w = a, status 0
__global__ void eig1_kernel(const double* A, double* Z, double* w, int* status) {
  w[0] = A[0];
  Z[0] = 1.0;
  status[0] = 0;
}

// S = (A + A^T) / 2 (n x n)
__global__ void symmetrize_copy_kernel(int n, const double* __restrict__ A, int lda,
                                       double* __restrict__ S, int lds) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  S[i + (int64_t)j * lds] = 0.5 * (A[i + (int64_t)j * lda] + A[j + (int64_t)i * lda]);
}

__global__ void copy_block_cm_kernel(int rows, int cols, const double* __restrict__ S, int lds,
                                     double* __restrict__ D, int ldd, double scale) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  D[i + (int64_t)j * ldd] = scale * S[i + (int64_t)j * lds];
}

// X(i, j) *= r[i] (row scaling), optionally adding Add(i, j) for i < add_rows first
__global__ void scale_rows_add_kernel(int rows, int cols, const double* __restrict__ r,
                                      double* __restrict__ X, int ldx, const double* __restrict__ Add,
                                      int ldadd, int add_rows) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  double x = X[i + (int64_t)j * ldx];
  if (Add && i < add_rows) x += Add[i + (int64_t)j * ldadd];
  X[i + (int64_t)j * ldx] = r ? r[i] * x : x;
}

// d_i = G_ii^-1/2 (0 for a zero column); MB = D GB D, MA = D GA D (both
// symmetrised).  GA may be null (only MB).
__global__ void dscale2_kernel(int n, const double* __restrict__ GB, int ldb,
                               const double* __restrict__ GA, int lda, double* __restrict__ d,
                               double* __restrict__ MB, double* __restrict__ MA, int ldm) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  const double gi = GB[i + (int64_t)i * ldb], gj = GB[j + (int64_t)j * ldb];
  const double di = gi > DBL_MIN ? 1.0 / sqrt(gi) : 0.0, dj = gj > DBL_MIN ? 1.0 / sqrt(gj) : 0.0;
  if (j == 0) d[i] = di;
  MB[i + (int64_t)j * ldm] = di * (0.5 * (GB[i + (int64_t)j * ldb] + GB[j + (int64_t)i * ldb])) * dj;
  if (GA)
    MA[i + (int64_t)j * ldm] =
        di * (0.5 * (GA[i + (int64_t)j * lda] + GA[j + (int64_t)i * lda])) * dj;
}

// The congruence T1^T M T1, T1 = blkdiag(Y11, I), of the scaled explicit
// pencil (MB, MA), completed from the blocks the GEMMs wrote: SB' has the
// identity on its leading o x o block, Fb = Y11^T MB[0:o, o:] above and its
// transpose below the diagonal, MB on the trailing block; SA' has the GEMM's
// leading block, Ka[:, o:] = Y11^T MA[0:o, o:] off the diagonal and MA on the
// trailing block.  Both come out with both triangles.
__global__ void pre_fill_kernel(int ns, int o, const double* __restrict__ MB,
                                const double* __restrict__ MA, int ldm,
                                const double* __restrict__ Ka, int ldk, double* __restrict__ SB,
                                double* __restrict__ SA, int lds) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ns * ns) return;
  const int i = (int)(e % ns), j = (int)(e / ns);
  if (i < o && j < o) {  // SA' leading block comes from its GEMM
    SB[i + (int64_t)j * lds] = i == j ? 1.0 : 0.0;
  } else if (i < o) {    // SB' upper off-diagonal block comes from its GEMM
    SA[i + (int64_t)j * lds] = Ka[i + (int64_t)j * ldk];
  } else if (j < o) {
    SB[i + (int64_t)j * lds] = SB[j + (int64_t)i * lds];
    SA[i + (int64_t)j * lds] = Ka[j + (int64_t)i * ldk];
  } else {
    SB[i + (int64_t)j * lds] = MB[i + (int64_t)j * ldm];
    SA[i + (int64_t)j * lds] = MA[i + (int64_t)j * ldm];
  }
}

// C(i, j) = d_i (i < o ? Ct(i, j) : C(i, j)): the coefficients in the basis
// S back from the congruence, C = D blkdiag(Y11, I) C'.
__global__ void pre_back_kernel(int ns, int m, int o, const double* __restrict__ d,
                                const double* __restrict__ Ct, int ldt, double* __restrict__ C,
                                int ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ns * m) return;
  const int i = (int)(e % ns), j = (int)(e / ns);
  const double x = i < o ? Ct[i + (int64_t)j * ldt] : C[i + (int64_t)j * ldc];
  C[i + (int64_t)j * ldc] = d[i] * x;
}

// H (ns x ns): H[0:o, 0:o] = MA[0:o, 0:o]; H[0:o, o:] = Qm[0:o, :] and its
// transpose below; H[o:, o:] is written by a GEMM.
__global__ void assemble_h_kernel(int ns, int o, const double* __restrict__ MA, int ldm,
                                  const double* __restrict__ Qm, int ldq, double* __restrict__ H,
                                  int ldh) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ns * ns) return;
  const int i = (int)(e % ns), j = (int)(e / ns);
  if (i >= o && j >= o) return;
  double v;
  if (i < o && j < o) v = MA[i + (int64_t)j * ldm];
  else if (i < o) v = Qm[i + (int64_t)(j - o) * ldq];
  else v = Qm[j + (int64_t)(i - o) * ldq];
  H[i + (int64_t)j * ldh] = v;
}

// cond(R) of R = [[I, F], [0, Rw]] (o + nw = ns; o = 0: R = Rw) from 8 power
// iterations on M = R^T R = MB and 8 on R^-1 R^-T = MB^-1, with R^-1 =
// [[I, Yt], [0, Yw]] given by its last nw columns Y (ns x nw); FP32 in shared
// memory (the value feeds an order-of-magnitude test).  out[0] = cond(R),
// inf when a factor is non-finite; skip: no-op when *skip != 0 (then out[0]
// is set to inf).
__global__ void __launch_bounds__(1024, 1) cond_struct_kernel(int ns, int o, const double* __restrict__ MB,
                                                              int ldm, const double* __restrict__ Y,
                                                              int ldy, double* out, const int* skip) {
  if (skip && *skip) {
    if (threadIdx.x == 0) out[0] = INFINITY;
    return;
  }
  extern __shared__ float cs[];
  const int nw = ns - o;
  float* F = cs;               // o x nw   (MB[0:o, o:])
  float* Bw = F + o * nw;      // nw x nw  (MB[o:, o:])
  float* Yt = Bw + nw * nw;    // o x nw
  float* Yw = Yt + o * nw;     // nw x nw
  float* x = Yw + nw * nw;     // ns
  float* y = x + ns;           // ns
  float* z = y + ns;           // ns
  __shared__ float red[3][32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int e = t; e < o * nw; e += blockDim.x) {
    const int i = e % o, j = e / o;
    F[e] = (float)MB[i + (int64_t)(o + j) * ldm];
    Yt[e] = (float)Y[i + (int64_t)j * ldy];
  }
  for (int e = t; e < nw * nw; e += blockDim.x) {
    const int i = e % nw, j = e / nw;
    Bw[e] = (float)MB[(o + i) + (int64_t)(o + j) * ldm];
    Yw[e] = (float)Y[(o + i) + (int64_t)j * ldy];
  }
  __syncthreads();
  auto sum3 = [&](float a, float b, float c, float& ra, float& rb, float& rc) {
    for (int q = 16; q > 0; q >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, q);
      b += __shfl_xor_sync(0xffffffffu, b, q);
      c += __shfl_xor_sync(0xffffffffu, c, q);
    }
    if (lane == 0) {
      red[0][warp] = a;
      red[1][warp] = b;
      red[2][warp] = c;
    }
    __syncthreads();
    ra = rb = rc = 0.f;
    for (int w = 0; w < 32; ++w) {
      ra += red[0][w];
      rb += red[1][w];
      rc += red[2][w];
    }
    __syncthreads();
  };
  // out = MB in:  top = in_top + F in_w;  w = F^T in_top + Bw in_w
  auto mb_apply = [&](const float* in, float* res) {
    for (int i = t; i < ns; i += blockDim.x) {
      float s = 0.f;
      if (i < o) {
        s = in[i];
        for (int j = 0; j < nw; ++j) s = fmaf(F[i + j * o], in[o + j], s);
      } else {
        const int iw = i - o;
        for (int j = 0; j < o; ++j) s = fmaf(F[j + iw * o], in[j], s);
        for (int j = 0; j < nw; ++j) s = fmaf(Bw[iw + j * nw], in[o + j], s);
      }
      res[i] = s;
    }
    __syncthreads();
  };
  // res = R^-T in: top = in_top; w = Yt^T in_top + Yw^T in_w
  auto rit_apply = [&](const float* in, float* res) {
    for (int i = t; i < ns; i += blockDim.x) {
      float s;
      if (i < o) {
        s = in[i];
      } else {
        const int iw = i - o;
        s = 0.f;
        for (int j = 0; j < o; ++j) s = fmaf(Yt[j + iw * o], in[j], s);
        for (int j = 0; j < nw; ++j) s = fmaf(Yw[j + iw * nw], in[o + j], s);
      }
      res[i] = s;
    }
    __syncthreads();
  };
  // res = R^-1 in: top = in_top + Yt in_w; w = Yw in_w
  auto ri_apply = [&](const float* in, float* res) {
    for (int i = t; i < ns; i += blockDim.x) {
      float s = i < o ? in[i] : 0.f;
      if (i < o) {
        for (int j = 0; j < nw; ++j) s = fmaf(Yt[i + j * o], in[o + j], s);
      } else {
        const int iw = i - o;
        for (int j = 0; j < nw; ++j) s = fmaf(Yw[iw + j * nw], in[o + j], s);
      }
      res[i] = s;
    }
    __syncthreads();
  };
  auto power = [&](int which) -> float {
    for (int i = t; i < ns; i += blockDim.x) x[i] = 1.0f + 0.001f * (float)(i % 7);
    __syncthreads();
    float lam = 0.f;
    for (int it = 0; it < 8; ++it) {
      float* res = y;
      if (which == 0) {
        mb_apply(x, y);
      } else {
        rit_apply(x, y);
        ri_apply(y, z);
        res = z;
      }
      float a = 0.f, b = 0.f, c = 0.f;
      for (int i = t; i < ns; i += blockDim.x) {
        a += x[i] * res[i];
        b += res[i] * res[i];
        c += x[i] * x[i];
      }
      float xy, yy, xx;
      sum3(a, b, c, xy, yy, xx);
      if (!(yy > 0.f) || !isfinite(yy)) return INFINITY;
      if (xx > 0.f) lam = fmaxf(lam, xy / xx);
      const float inv = rsqrtf(yy);
      for (int i = t; i < ns; i += blockDim.x) x[i] = res[i] * inv;
      __syncthreads();
    }
    return lam;
  };
  const float lmax = power(0);
  const float imax = power(1);
  if (t == 0)
    out[0] = (isfinite(lmax) && isfinite(imax) && lmax > 0.f && imax > 0.f)
                 ? sqrt((double)lmax * (double)imax)
                 : INFINITY;
}

// Q2(i, j) = th[i] * Q(i, j)
__global__ void scale_rows_by_kernel(int rows, int cols, const double* __restrict__ th,
                                     const double* __restrict__ Q, int ldq, double* __restrict__ Q2,
                                     int ldq2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  Q2[i + (int64_t)j * ldq2] = th[i] * Q[i + (int64_t)j * ldq];
}

// svqb / svqbDrop transform (Algorithms 4, 6) from the eigenpairs (w ascending,
// Z) of D G D: keep J = {j : w_j > tau max|w|} (drop) or all with w clamped
// at tau max|w| (replace); T(:, t) = d .* Z(:, first + t) / sqrt(w); nkeep[0]
// is the kept count.  One CTA computes the split, all threads fill T.
__global__ void svqb_dev_kernel(int nu, const double* __restrict__ w, const double* __restrict__ d,
                                const double* __restrict__ Z, int ldz, int drop, double tau,
                                double* __restrict__ T, int ldt, int* nkeep) {
  __shared__ int s_first;
  __shared__ double s_floor;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < nu; ++i) mx = fmax(mx, fabs(w[i]));
    int first = 0;
    double floor_ = -INFINITY;
    if (!(mx > 0.0)) {
      first = nu;
    } else if (drop) {
      while (first < nu && !(w[first] > tau * mx)) ++first;
    } else {
      floor_ = tau * mx;
    }
    s_first = first;
    s_floor = floor_;
    nkeep[0] = nu - first;
  }
  __syncthreads();
  const int first = s_first, keep = nu - first;
  for (int e = threadIdx.x; e < nu * keep; e += blockDim.x) {
    const int i = e % nu, c = e / nu;
    const double th = fmax(w[first + c], s_floor);
    T[i + (int64_t)c * ldt] = d[i] * Z[i + (int64_t)(first + c) * ldz] / sqrt(th);
  }
}

// D = diag(w[0:n]) (n x n, leading dimension ldd)
__global__ void diag_matrix_kernel(int n, const double* __restrict__ w, double* __restrict__ D,
                                   int ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  D[i + (int64_t)j * ldd] = i == j ? w[i] : 0.0;
}

unsigned nblk(int64_t total) { return (unsigned)std::max<int64_t>(1, ceil_div(total, 256)); }

}  // namespace

// ==================================================================== host

int DevDense::init(int64_t nmax_) {
  nmax = (int)std::min<int64_t>(nmax_, kDevDenseMax);
  const size_t nn = (size_t)nmax * nmax;
  const int tiles = (int)(ceil_div(nmax, kGT) * ceil_div(2 * nmax, kGT));
  auto g = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    bufs.push_back(*p);
    return true;
  };
  bool ok = true;
  for (double** b : {&X, &X1, &E, &Zt, &T1, &T2, &T3, &T4}) ok = ok && g((void**)b, nn * sizeof(double));
  ok = ok && g((void**)&XA, 2 * nn * sizeof(double));   // [X | A X]
  ok = ok && g((void**)&GS, 2 * nn * sizeof(double));   // [G | S]
  ok = ok && g((void**)&V32, nn * sizeof(float));
  ok = ok && g((void**)&Y32, nn * sizeof(float));
  ok = ok && g((void**)&f32v, 4 * (size_t)nmax * sizeof(float));
  ok = ok && g((void**)&vec, (8 * (size_t)nmax + 256) * sizeof(double));
  ok = ok && g((void**)&scal, 16 * sizeof(double));
  ok = ok && g((void**)&ints, (4 * (size_t)nmax + 64) * sizeof(int));
  ok = ok && g((void**)&part, (size_t)tiles * kMaxKs * 256 * sizeof(double));
  ok = ok && g((void**)&cnt, (size_t)tiles * sizeof(unsigned));
  if (!ok) return LOBPCG_ERR_OOM;
  cnt_tiles = tiles;
  if (cudaMemset(cnt, 0, (size_t)tiles * sizeof(unsigned)) != cudaSuccess) return LOBPCG_ERR_CUDA;
  if (cudaMemset(ints, 0, (4 * (size_t)nmax + 64) * sizeof(int)) != cudaSuccess)
    return LOBPCG_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return LOBPCG_ERR_CUDA;
  return LOBPCG_OK;
}

void DevDense::release() {
  for (void* p : bufs) cudaFree(p);
  bufs.clear();
  nmax = 0;
}

int dev_gemm(DenseLayer& L, bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
             int lda, const double* B, int ldb, double beta, const double* Cin, int ldcin,
             double* C, int ldc, const int* skip) {
  if (m <= 0 || n <= 0) return LOBPCG_OK;
  DevDense& D = L.dev;
  const int tiles = (int)(ceil_div(m, kGT) * ceil_div(n, kGT));
  if (tiles > D.cnt_tiles) return LOBPCG_ERR_ARG;
  const int kchunks = (int)std::max<int64_t>(1, ceil_div(k, kGK));
  int ks = (int)std::min<int64_t>(std::min<int64_t>(kMaxKs, kchunks),
                                  std::max<int64_t>(1, ceil_div(2 * 152, tiles)));
  const int kper = (int)(ceil_div(kchunks, ks) * kGK);
  ks = (int)ceil_div(std::max(k, 1), kper);
  if (!Cin) {
    Cin = C;
    ldcin = ldc;
  }
  gemm64_kernel<<<dim3((unsigned)tiles, (unsigned)ks), 256, 0, L.st>>>(
      m, n, k, ta ? 1 : 0, tb ? 1 : 0, alpha, A, lda, B, ldb, beta, Cin, ldcin, C, ldc, ks, kper,
      D.part, D.cnt, skip);
  DLAUNCH(L);
  return LOBPCG_OK;
}

int dev_chol(DenseLayer& L, int n, double* A, int lda, int* info) {
  if (n > kCholMax) return LOBPCG_ERR_ARG;
  const size_t sh = (size_t)n * n * sizeof(double);
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    LOB_CUDA_OK(cudaFuncSetAttribute(chol64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kCholMax * kCholMax * 8));
    LOB_CUDA_OK(cudaFuncSetAttribute(trinv64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kCholMax * kCholMax * 8));
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  chol64_kernel<<<1, 256, sh, L.st>>>(n, A, lda, info);
  DLAUNCH(L);
  return LOBPCG_OK;
}

int dev_trinv(DenseLayer& L, int n, const double* R, int ldr, double* X, int ldx, const int* skip) {
  if (n > kCholMax) return LOBPCG_ERR_ARG;
  trinv64_kernel<<<1, 256, (size_t)n * n * sizeof(double), L.st>>>(n, R, ldr, X, ldx, skip);
  DLAUNCH(L);
  return LOBPCG_OK;
}

// Eigendecomposition of the symmetric n x n FP64 matrix A (column-major, not
// modified): Z (n x n, ldz) orthonormal eigenvectors, w ascending; status
// (device int) 0 on success, 1 when the refinement's check failed (the caller
// falls back).  n <= kDevDenseMax.
int dev_syev(DenseLayer& L, int n, const double* A, int lda, double* Z, int ldz, double* w,
             int* status) {
  DevDense& D = L.dev;
  if (n > D.nmax || n > kDevDenseMax) return LOBPCG_ERR_ARG;
  int dev = 0;
  cudaGetDevice(&dev);
  static bool configured[64] = {false};
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    LOB_CUDA_OK(cudaFuncSetAttribute(tridiag32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kDevDenseMax * (kDevDenseMax + 1) / 2 * 4));
    LOB_CUDA_OK(cudaFuncSetAttribute(tridiag32_full_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kTridFull * (kTridFull | 1) * 4));
    LOB_CUDA_OK(cudaFuncSetAttribute(tridiag_eig_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (3 * kDevDenseMax + 6 * 32 * kDevDenseMax) * 4));
    LOB_CUDA_OK(cudaFuncSetAttribute(backtransform_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (kDevDenseMax * (kDevDenseMax - 1) / 2 + 16 * kDevDenseMax) * 4));
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  if (n == 1) {
    eig1_kernel<<<1, 1, 0, L.st>>>(A, Z, w, status);
    DLAUNCH(L);
    return LOBPCG_OK;
  }
  float* d32 = D.f32v;
  float* e32 = D.f32v + D.nmax;
  float* tau32 = D.f32v + 2 * D.nmax;
  float* lam32 = D.f32v + 3 * D.nmax;
  double* normA = D.scal;  // scal[0] = ||A||_F
  // the refinement multiplies by the symmetric part of A (a projected
  // matrix formed by products is symmetric only to rounding)
  symmetrize_copy_kernel<<<nblk((int64_t)n * n), 256, 0, L.st>>>(n, A, lda, D.Zt, n);
  DLAUNCH(L);
  A = D.Zt;
  lda = n;
  if (n <= kTridFull)
    tridiag32_full_kernel<<<1, 1024, (size_t)n * (n | 1) * 4, L.st>>>(n, A, lda, d32, e32, D.V32,
                                                                      n, tau32, normA);
  else
    tridiag32_kernel<<<1, 1024, (size_t)n * (n + 1) / 2 * 4, L.st>>>(n, A, lda, d32, e32, D.V32,
                                                                     n, tau32, normA);
  DLAUNCH(L);
  bisect_kernel<<<(unsigned)ceil_div(4 * n, 256), 256, 0, L.st>>>(n, d32, e32, lam32);
  DLAUNCH(L);
  tridiag_eig_kernel<<<(unsigned)ceil_div(n, 32), 32, (size_t)(3 * n + 6 * 32 * n) * 4, L.st>>>(
      n, d32, e32, lam32, D.Y32, n);
  DLAUNCH(L);
  cluster_orth_kernel<<<1, 1024, 0, L.st>>>(n, lam32, D.Y32, n);
  DLAUNCH(L);
  // X (first n columns of XA) = Q Y
  double* X = D.XA;
  backtransform_kernel<<<(unsigned)ceil_div(n, 16), 256,
                         (size_t)((n * (n - 1)) / 2 + 16 * n) * 4, L.st>>>(
      n, D.V32, n, tau32, D.Y32, n, X, n);
  DLAUNCH(L);
  return dev_syev_refine(L, n, Z, ldz, w, status, kRefSteps);
}

// Refinement of the current X (first block of D.XA) against the symmetric A
// kept in D.Zt: `steps` Ogita-Aishima steps, two Newton-Schulz steps, the
// final products, the finalize pass, the permutation into Z and Jacobi on
// the coupled runs.  Also the second chance after a failed check: more
// steps from where the first call stopped.
int dev_syev_refine(DenseLayer& L, int n, double* Z, int ldz, double* w, int* status, int steps) {
  DevDense& D = L.dev;
  const double* A = D.Zt;
  const int lda = n;
  double* normA = D.scal;
  double* delta = D.scal + 1;
  int* perm = D.ints + 4;
  int* runs = perm + D.nmax;
  int* nruns = runs + 2 * D.nmax;
  // skip flags of the steps (flag[s] for step s) and the largest correction
  // of each step
  if (steps > 16) return LOBPCG_ERR_ARG;
  int* flag = D.ints + 4 * D.nmax + 24;
  // (D.vec: the norm partials at 0 .. 127, d at 128 .. 128 + n, then these)
  unsigned long long* emax = reinterpret_cast<unsigned long long*>(D.vec + 136 + D.nmax);
  double* X = D.XA;
  double* AX = D.XA + (size_t)n * n;
  double* G = D.GS;
  LOB_CUDA_OK(cudaMemsetAsync(flag, 0, (steps + 1) * sizeof(int), L.st));
  LOB_CUDA_OK(cudaMemsetAsync(emax, 0, steps * sizeof(unsigned long long), L.st));
  int rc;
  for (int s = 0; s < steps; ++s) {
    int* done = flag + s;
    // [G, S] = X^T [X, A X]
    if ((rc = dev_gemm(L, false, false, n, n, n, 1.0, A, lda, X, n, 0.0, nullptr, 0, AX, n, done)))
      return rc;
    if ((rc = dev_gemm(L, true, false, n, 2 * n, n, 1.0, X, n, D.XA, n, 0.0, nullptr, 0, G, n,
                       done)))
      return rc;
    oa_norms_kernel<<<kOaBlocks, 256, 0, L.st>>>(n, D.GS, D.vec, D.vec + 2 * kOaBlocks, done);
    DLAUNCH(L);
    oa_e_kernel<<<nblk((int64_t)n * n), 256, 0, L.st>>>(n, D.GS, D.vec, D.vec + 2 * kOaBlocks,
                                                        normA, D.E, done, delta, emax + s);
    DLAUNCH(L);
    oa_next_kernel<<<1, 32, 0, L.st>>>(done, emax + s, flag + s + 1);
    DLAUNCH(L);
    // X1 = X + X E
    if ((rc = dev_gemm(L, false, false, n, n, n, 1.0, X, n, D.E, n, 1.0, X, n, D.X1, n, done)))
      return rc;
    // X = X1 (skipped with the step)
    copy_skip_kernel<<<nblk((int64_t)n * n), 256, 0, L.st>>>(n, n, D.X1, n, X, n, done);
    DLAUNCH(L);
  }
  // two Newton-Schulz steps X = X (3/2 I - 1/2 X^T X): the last first-order
  // step leaves ||I - X^T X|| up to ~1e-4 on pairs it has just separated;
  // each step squares it
  for (int s = 0; s < 2; ++s) {
    if ((rc = dev_gemm(L, true, false, n, n, n, 1.0, X, n, X, n, 0.0, nullptr, 0, G, n, nullptr)))
      return rc;
    if ((rc = dev_gemm(L, false, false, n, n, n, -0.5, X, n, G, n, 1.5, X, n, D.X1, n, nullptr)))
      return rc;
    copy_block_cm_kernel<<<nblk((int64_t)n * n), 256, 0, L.st>>>(n, n, D.X1, n, X, n, 1.0);
    DLAUNCH(L);
  }
  // final [G, S] = X^T [X, A X]
  if ((rc = dev_gemm(L, false, false, n, n, n, 1.0, A, lda, X, n, 0.0, nullptr, 0, AX, n, nullptr)))
    return rc;
  if ((rc = dev_gemm(L, true, false, n, 2 * n, n, 1.0, X, n, D.XA, n, 0.0, nullptr, 0, G, n,
                     nullptr)))
    return rc;
  eig_finalize_kernel<<<1, 1024, 0, L.st>>>(n, D.GS, normA, perm, runs, nruns, w, status);
  DLAUNCH(L);
  permute_cols_dev_kernel<<<nblk((int64_t)n * n), 256, 0, L.st>>>(n, X, n, perm, Z, ldz);
  DLAUNCH(L);
  run_jacobi_kernel<<<(unsigned)std::max(1, n / 2), 256, 0, L.st>>>(n, D.GS, perm, runs, nruns, Z,
                                                                     ldz, w);
  DLAUNCH(L);
  return LOBPCG_OK;
}

// Thin orthonormal basis of the span of the tall M (m x c, m > c) into Q
// (m x c, ldq): FP32 Householder QR, then two FP64 Newton-Schulz steps.
int dev_orth_basis(DenseLayer& L, int m, int c, const double* M, int ldm, double* Q, int ldq) {
  DevDense& D = L.dev;
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    LOB_CUDA_OK(cudaFuncSetAttribute(qr32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     200 * 1024));
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  const size_t sh = 2 * (size_t)m * c * sizeof(float);
  if (sh > 200 * 1024 || c > 256) return LOBPCG_ERR_ARG;
  qr32_kernel<<<1, 1024, sh, L.st>>>(m, c, M, ldm, Q, ldq);
  DLAUNCH(L);
  int rc;
  for (int s = 0; s < 2; ++s) {
    if ((rc = dev_gemm(L, true, false, c, c, m, 1.0, Q, ldq, Q, ldq, 0.0, nullptr, 0, D.T4, c,
                       nullptr)))
      return rc;
    if ((rc = dev_gemm(L, false, false, m, c, c, -0.5, Q, ldq, D.T4, c, 1.5, Q, ldq, D.T3, m,
                       nullptr)))
      return rc;
    copy_block_cm_kernel<<<nblk((int64_t)m * c), 256, 0, L.st>>>(m, c, D.T3, m, Q, ldq, 1.0);
    DLAUNCH(L);
  }
  return LOBPCG_OK;
}

// --------------------------------------------- Rayleigh-Ritz, device path

// The device path takes a projected pencil when every piece fits its
// one-CTA kernels: order <= 256 (eigensolver), Cholesky factors of order
// <= 160, the cond(R) estimate's FP32 copies and the C_p QR in shared memory.
bool dev_rr_fits(const DenseLayer& L, int ns, int nx, int nw) {
  if (L.eig_mode != 0 || ns > L.dev.nmax || ns > kDevDenseMax) return false;
  if (nw > kCholMax || nx > kCholMax) return false;
  const int o = ns - nw;
  const size_t cond_sh = (size_t)(2 * o * nw + 2 * nw * nw + 3 * ns) * 4;
  const size_t qr_sh = 2 * (size_t)(ns - nx) * nx * 4;
  return cond_sh <= 200 * 1024 && qr_sh <= 200 * 1024;
}

int syevd_fallback(DenseLayer& L, int n, double* A, int lda) {
  ++L.dev_fallbacks;
  if (cusolverDnDsyevd(L.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A, lda, L.ev,
                       L.work, L.lwork, L.info) != CUSOLVER_STATUS_SUCCESS)
    return LOBPCG_ERR_CUDA;
  return LOBPCG_OK;
}

namespace {

int configure_cond(DenseLayer& L) {
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    LOB_CUDA_OK(cudaFuncSetAttribute(cond_struct_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  (void)L;
  return LOBPCG_OK;
}

// read n_ints device ints (from ints) and n_dbl device doubles (from dbl) in
// one host wait
int read_flags(DenseLayer& L, const int* ints, int n_ints, const double* dbl, int n_dbl,
               int* ih, double* dh) {
  if (n_ints) LOB_CUDA_OK(cudaMemcpyAsync(L.host, ints, n_ints * sizeof(int), cudaMemcpyDeviceToHost, L.st));
  if (n_dbl)
    LOB_CUDA_OK(cudaMemcpyAsync(L.host + 8, dbl, n_dbl * sizeof(double), cudaMemcpyDeviceToHost, L.st));
  LOB_CUDA_OK(cudaStreamSynchronize(L.st));
  ++L.syncs;
  if (n_ints) memcpy(ih, L.host, n_ints * sizeof(int));
  if (n_dbl) memcpy(dh, L.host + 8, n_dbl * sizeof(double));
  return LOBPCG_OK;
}

// count the reasons of a failed check of the device eigensolver
void note_check(DenseLayer& L, int mask) {
  if (mask & 1) ++L.check_fail[0];
  if (mask & 2) ++L.check_fail[1];
  if (mask & 8) ++L.check_fail[2];
}

// Eigenvectors Z of H (order n) with eigenvalues in L.ev: device eigensolver,
// its status read back with the other flags by the caller.
int eig_into(DenseLayer& L, int n, const double* H, double* Z, int* status) {
  ++L.dev_calls;
  return dev_syev(L, n, H, n, Z, n, L.ev, status);
}

// After a failed check: when only the coupled groups were too wide, three
// more refinement steps from where the first call stopped (one more host
// read); otherwise, or when that fails too, cuSOLVER on a copy of H.
int eig_recover(DenseLayer& L, int n, const double* H, double* Z, int mask) {
  int rc;
  if (mask == 2) {
    int* est = L.dev.ints + 2;
    if ((rc = dev_syev_refine(L, n, Z, n, L.ev, est, 3))) return rc;
    int fl = 0;
    LOB_CUDA_OK(cudaMemcpyAsync(L.host, est, sizeof(int), cudaMemcpyDeviceToHost, L.st));
    LOB_CUDA_OK(cudaStreamSynchronize(L.st));
    ++L.syncs;
    memcpy(&fl, L.host, sizeof(int));
    if (fl == 0) return LOBPCG_OK;
    note_check(L, fl);
  }
  copy_block_cm_kernel<<<nblk((int64_t)n * n), 256, 0, L.st>>>(n, n, H, n, Z, n, 1.0);
  DLAUNCH(L);
  return syevd_fallback(L, n, Z, n);
}


// C = [C_x, C_p] and the next P^T A P from T Z (ns x ns), Z and the
// eigenvalues L.ev (Algorithm 7, the LQ-based C_p of Sec. 4.2 restricted to
// the unlocked columns; an orthonormal basis of the span of
// M = Z_1perp^T Z_1(:, nc:nx) replaces the Householder Q of its LQ).
int rr_tail(DenseLayer& L, const double* TZ, const double* Z, int ns, int nx, int nc, double* C,
            int* npn_out, double* theta, double* PAP) {
  DevDense& D = L.dev;
  const int mrow = ns - nx, mcol = nx - nc;
  const int npn = std::min(mrow, mcol);
  int rc;
  copy_block_cm_kernel<<<nblk((int64_t)ns * nx), 256, 0, L.st>>>(ns, nx, TZ, ns, C, ns, 1.0);
  DLAUNCH(L);
  if (npn > 0) {
    if (mcol >= mrow) {  // M spans the whole (ns - nx)-dimensional space: Q = I
      copy_block_cm_kernel<<<nblk((int64_t)ns * mrow), 256, 0, L.st>>>(
          ns, mrow, TZ + (int64_t)nx * ns, ns, C + (int64_t)nx * ns, ns, 1.0);
      DLAUNCH(L);
      diag_matrix_kernel<<<nblk((int64_t)npn * npn), 256, 0, L.st>>>(npn, L.ev + nx, PAP, npn);
      DLAUNCH(L);
    } else {
      double* M = D.Zt;
      double* Q = D.E;
      double* Q2 = D.X;
      if ((rc = dev_gemm(L, true, false, mrow, mcol, nx, 1.0, Z + (int64_t)nx * ns, ns,
                         Z + (int64_t)nc * ns, ns, 0.0, nullptr, 0, M, mrow, nullptr)))
        return rc;
      if ((rc = dev_orth_basis(L, mrow, mcol, M, mrow, Q, mrow))) return rc;
      if ((rc = dev_gemm(L, false, false, ns, mcol, mrow, 1.0, TZ + (int64_t)nx * ns, ns, Q, mrow,
                         0.0, nullptr, 0, C + (int64_t)nx * ns, ns, nullptr)))
        return rc;
      scale_rows_by_kernel<<<nblk((int64_t)mrow * mcol), 256, 0, L.st>>>(mrow, mcol, L.ev + nx, Q,
                                                                          mrow, Q2, mrow);
      DLAUNCH(L);
      if ((rc = dev_gemm(L, true, false, mcol, mcol, mrow, 1.0, Q, mrow, Q2, mrow, 0.0, nullptr, 0,
                         PAP, npn, nullptr)))
        return rc;
    }
  }
  LOB_CUDA_OK(cudaMemcpyAsync(theta, L.ev, nx * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
  *npn_out = npn;
  return LOBPCG_OK;
}

}  // namespace

// Algorithm 2 on the Gram pair (GA, GB), device path.
int rr_initial_dev(DenseLayer& L, const double* GA, const double* GB, int nx, double* C,
                   double* theta, bool* breakdown) {
  DevDense& D = L.dev;
  *breakdown = false;
  double* MB = L.A[0];
  double* MA = L.A[1];
  double* H = L.A[2];
  double* Z = L.A[3];
  double* Rf = D.T1;
  double* Ri = L.A[5];
  double* T = D.T2;
  int* info = D.ints + 1;
  int* est = D.ints + 2;
  double* cr = D.scal + 2;
  int rc;
  if ((rc = configure_cond(L))) return rc;
  LOB_CUDA_OK(cudaMemsetAsync(info, 0, 2 * sizeof(int), L.st));
  dscale2_kernel<<<nblk((int64_t)nx * nx), 256, 0, L.st>>>(nx, GB, nx, GA, nx, L.d, MB, MA, nx);
  DLAUNCH(L);
  copy_block_cm_kernel<<<nblk((int64_t)nx * nx), 256, 0, L.st>>>(nx, nx, MB, nx, Rf, nx, 1.0);
  DLAUNCH(L);
  if ((rc = dev_chol(L, nx, Rf, nx, info))) return rc;
  if ((rc = dev_trinv(L, nx, Rf, nx, Ri, nx, info))) return rc;
  cond_struct_kernel<<<1, 1024, (size_t)(2 * nx * nx + 3 * nx) * 4, L.st>>>(nx, 0, MB, nx, Ri, nx,
                                                                            cr, info);
  DLAUNCH(L);
  // H = Ri^T MA Ri
  if ((rc = dev_gemm(L, false, false, nx, nx, nx, 1.0, MA, nx, Ri, nx, 0.0, nullptr, 0, T, nx, info)))
    return rc;
  if ((rc = dev_gemm(L, true, false, nx, nx, nx, 1.0, Ri, nx, T, nx, 0.0, nullptr, 0, H, nx, info)))
    return rc;
  if ((rc = eig_into(L, nx, H, Z, est))) return rc;
  int fl[2];
  double condR;
  if ((rc = read_flags(L, info, 2, cr, 1, fl, &condR))) return rc;
  // breakdown: Cholesky failed or D X0^T B X0 D = R^T R is numerically
  // singular, cond(R)^2 >= 1 / (n_x eps)
  if (fl[0] != 0 || !(condR * condR < 1.0 / (nx * kEps64))) {
    *breakdown = true;
    return LOBPCG_OK;
  }
  note_check(L, fl[1]);
  if (fl[1] != 0 && (rc = eig_recover(L, nx, H, Z, fl[1]))) return rc;
  // C = D Ri Z
  if ((rc = dev_gemm(L, false, false, nx, nx, nx, 1.0, Ri, nx, Z, nx, 0.0, nullptr, 0, C, nx,
                     nullptr)))
    return rc;
  scale_rows_add_kernel<<<nblk((int64_t)nx * nx), 256, 0, L.st>>>(nx, nx, L.d, C, nx, nullptr, 0, 0);
  DLAUNCH(L);
  LOB_CUDA_OK(cudaMemcpyAsync(theta, L.ev, nx * sizeof(double), cudaMemcpyDeviceToDevice, L.st));
  return LOBPCG_OK;
}

// Algorithm 7, device path.  With S = [X, P, W] and the identities (12)-(13),
// D S^T B S D = [[I, F], [F^T, Bw]] (F the o x n_w block of the X and P rows,
// o = n_x + n_p), so its Cholesky factor is R = [[I, F], [0, Rw]] with
// Rw^T Rw = Bw - F^T F, and R^-1 = [[I, Y_t], [0, Y_w]], Y_w = Rw^-1,
// Y_t = -F Y_w.  With MA = D S^T A S D and Y = R^-1(:, o:), the projected
// matrix H = R^-T MA R^-1 is MA on the first o rows and columns, Q = MA Y on
// the off-diagonal blocks and Y^T Q on the W block; T Z = D R^-1 Z =
// D ([Z_top; 0] + Y Z(o:, :)).
int rr_modified_dev(DenseLayer& L, const double* SAS, const double* SBS, int ns, int nx, int np,
                    int nc, bool use_ortho, double tau_skip, bool* flip, double* condR, double* C,
                    int* npn_out, double* theta, double* PAP) {
  DevDense& D = L.dev;
  *flip = false;
  *condR = 1.0;
  const int o = nx + np, nw = ns - o;
  double* MB = L.A[0];
  double* MA = L.A[1];
  double* H = L.A[2];
  double* Z = L.A[3];
  double* TZ = L.A[4];
  double* Y = L.A[5];  // ns x nw, leading dimension ns
  double* Sw = D.T1;   // nw x nw
  double* Qm = D.T2;   // ns x nw
  int* info = D.ints + 1;
  int* est = D.ints + 2;
  double* cr = D.scal + 2;
  int rc;
  if ((rc = configure_cond(L))) return rc;
  LOB_CUDA_OK(cudaMemsetAsync(info, 0, 2 * sizeof(int), L.st));
  if (use_ortho) {
    if ((rc = eig_into(L, ns, SAS, Z, est))) return rc;
    int fl[1];
    if ((rc = read_flags(L, est, 1, nullptr, 0, fl, nullptr))) return rc;
    note_check(L, fl[0]);
    if (fl[0] != 0 && (rc = eig_recover(L, ns, SAS, Z, fl[0]))) return rc;
    return rr_tail(L, Z, Z, ns, nx, nc, C, npn_out, theta, PAP);
  }
  dscale2_kernel<<<nblk((int64_t)ns * ns), 256, 0, L.st>>>(ns, SBS, ns, SAS, ns, L.d, MB, MA, ns);
  DLAUNCH(L);
  const double* Hsrc = MA;
  if (nw > 0) {
    const double* F = MB + (int64_t)o * ns;  // rows 0..o-1 of the W columns
    // Sw = Bw - F^T F
    if ((rc = dev_gemm(L, true, false, nw, nw, o, -1.0, F, ns, F, ns, 1.0,
                       MB + o + (int64_t)o * ns, ns, Sw, nw, nullptr)))
      return rc;
    if ((rc = dev_chol(L, nw, Sw, nw, info))) return rc;
    if ((rc = dev_trinv(L, nw, Sw, nw, Y + o, ns, info))) return rc;
    if ((rc = dev_gemm(L, false, false, o, nw, nw, -1.0, F, ns, Y + o, ns, 0.0, nullptr, 0, Y, ns,
                       info)))
      return rc;
    cond_struct_kernel<<<1, 1024, (size_t)(2 * o * nw + 2 * nw * nw + 3 * ns) * 4, L.st>>>(
        ns, o, MB, ns, Y, ns, cr, info);
    DLAUNCH(L);
    if ((rc = dev_gemm(L, false, false, ns, nw, ns, 1.0, MA, ns, Y, ns, 0.0, nullptr, 0, Qm, ns,
                       info)))
      return rc;
    assemble_h_kernel<<<nblk((int64_t)ns * ns), 256, 0, L.st>>>(ns, o, MA, ns, Qm, ns, H, ns);
    DLAUNCH(L);
    if ((rc = dev_gemm(L, true, false, nw, nw, ns, 1.0, Y, ns, Qm, ns, 0.0, nullptr, 0,
                       H + o + (int64_t)o * ns, ns, info)))
      return rc;
    Hsrc = H;
  } else {
    LOB_CUDA_OK(cudaMemsetAsync(cr, 0, sizeof(double), L.st));  // cond(I) = 1, set below
  }
  if ((rc = eig_into(L, ns, Hsrc, Z, est))) return rc;
  int fl[2];
  double c = 1.0;
  if ((rc = read_flags(L, info, 2, cr, 1, fl, &c))) return rc;
  if (nw == 0) c = 1.0;
  if (fl[0] != 0) {
    *flip = true;
    *condR = INFINITY;
    return LOBPCG_OK;
  }
  *condR = c;
  if (!(pow(c, -3.0) >= tau_skip)) {
    *flip = true;
    return LOBPCG_OK;
  }
  note_check(L, fl[1]);
  if (fl[1] != 0 && (rc = eig_recover(L, ns, Hsrc, Z, fl[1]))) return rc;
  // T Z = D ([Z_top; 0] + Y Z(o:, :))
  if (nw > 0) {
    if ((rc = dev_gemm(L, false, false, ns, ns, nw, 1.0, Y, ns, Z + o, ns, 0.0, nullptr, 0, TZ, ns,
                       nullptr)))
      return rc;
    scale_rows_add_kernel<<<nblk((int64_t)ns * ns), 256, 0, L.st>>>(ns, ns, L.d, TZ, ns, Z, ns, o);
  } else {
    copy_block_cm_kernel<<<nblk((int64_t)ns * ns), 256, 0, L.st>>>(ns, ns, Z, ns, TZ, ns, 1.0);
    DLAUNCH(L);
    scale_rows_add_kernel<<<nblk((int64_t)ns * ns), 256, 0, L.st>>>(ns, ns, L.d, TZ, ns, nullptr, 0, 0);
  }
  DLAUNCH(L);
  return rr_tail(L, TZ, Z, ns, nx, nc, C, npn_out, theta, PAP);
}

// The explicit Rayleigh-Ritz (every block of S^T A S and S^T B S computed,
// nothing taken from the identities (12)-(14)), device path.  With the
// scaling D = diag(S^T B S)^-1/2, MB = D S^T B S D and MA likewise, the
// leading o x o block (the X and P columns, o = n_x + n_p) is factored on its
// own, MB11 = R11^T R11, Y11 = R11^-1; the congruence T1 = blkdiag(Y11, I)
// turns the pencil into one whose B-block is [[I, Fb], [Fb^T, MB22]], which
// the structured path above factors (Cholesky of the Schur complement only).
// Together the two steps are the Cholesky factor of MB, R = [[R11, R11 Fb],
// [0, Rw]], so this is Algorithm 7 on the explicit pencil; the coefficients
// come back as C = D T1 C'.  The cond(R) estimate that drives the switch to
// orthogonalisation is that of the second factor: R11 is the factor of the
// Gram matrix of the previous iteration's B-orthonormal X and P, within
// rounding of the identity.  A failed R11 factorisation is a Cholesky
// failure (*flip, cond = inf), as in Algorithm 7.
bool dev_explicit_fits(const DenseLayer& L, int ns, int nx, int np) {
  const int o = nx + np;
  return o <= kCholMax && dev_rr_fits(L, ns, nx, ns - o);
}

int rr_explicit_dev(DenseLayer& L, const double* SAS, const double* SBS, int ns, int nx, int np,
                    int nc, double tau_skip, bool* flip, double* condR, double* C, int* npn_out,
                    double* theta, double* PAP) {
  DevDense& D = L.dev;
  *flip = false;
  *condR = 1.0;
  const int o = nx + np, nw = ns - o;
  // L.R[] hold the FP32-refinement blocks of dense_eig 1, unused on this path
  double* SB = L.R[0];   // ns x ns, T1^T MB T1
  double* SA = L.R[1];   // ns x ns, T1^T MA T1
  double* R11 = L.R[2];  // o x o, then kept as Y11 in Y
  double* Y = L.R[3];    // o x o, Y11
  double* d0 = L.R[4];   // ns
  double* Ka = L.R[5];   // o x ns, Y11^T MA[0:o, :]; then Y11 C'[0:o, :]
  double* MB = L.A[0];
  double* MA = L.A[1];
  int* info = D.ints + 4 * D.nmax + 16;
  int rc;
  dscale2_kernel<<<nblk((int64_t)ns * ns), 256, 0, L.st>>>(ns, SBS, ns, SAS, ns, d0, MB, MA, ns);
  DLAUNCH(L);
  copy_block_cm_kernel<<<nblk((int64_t)o * o), 256, 0, L.st>>>(o, o, MB, ns, R11, o, 1.0);
  DLAUNCH(L);
  LOB_CUDA_OK(cudaMemsetAsync(info, 0, sizeof(int), L.st));
  if ((rc = dev_chol(L, o, R11, o, info))) return rc;
  int fl = 0;
  LOB_CUDA_OK(cudaMemcpyAsync(L.host, info, sizeof(int), cudaMemcpyDeviceToHost, L.st));
  LOB_CUDA_OK(cudaStreamSynchronize(L.st));
  ++L.syncs;
  memcpy(&fl, L.host, sizeof(int));
  if (fl != 0) {
    *flip = true;
    *condR = INFINITY;
    return LOBPCG_OK;
  }
  if ((rc = dev_trinv(L, o, R11, o, Y, o, nullptr))) return rc;
  // Ka = Y11^T MA[0:o, :], SA'11 = Ka[:, 0:o] Y11, SB'12 = Y11^T MB[0:o, o:]
  if ((rc = dev_gemm(L, true, false, o, ns, o, 1.0, Y, o, MA, ns, 0.0, nullptr, 0, Ka, o,
                     nullptr)))
    return rc;
  if ((rc = dev_gemm(L, false, false, o, o, o, 1.0, Ka, o, Y, o, 0.0, nullptr, 0, SA, ns,
                     nullptr)))
    return rc;
  if (nw > 0 && (rc = dev_gemm(L, true, false, o, nw, o, 1.0, Y, o, MB + (int64_t)o * ns, ns, 0.0,
                               nullptr, 0, SB + (int64_t)o * ns, ns, nullptr)))
    return rc;
  pre_fill_kernel<<<nblk((int64_t)ns * ns), 256, 0, L.st>>>(ns, o, MB, MA, ns, Ka, o, SB, SA, ns);
  DLAUNCH(L);
  int npn = 0;
  if ((rc = rr_modified_dev(L, SA, SB, ns, nx, np, nc, false, tau_skip, flip, condR, C, &npn,
                            theta, PAP)))
    return rc;
  if (*flip) return LOBPCG_OK;
  const int m = nx + npn;
  if ((rc = dev_gemm(L, false, false, o, m, o, 1.0, Y, o, C, ns, 0.0, nullptr, 0, Ka, o, nullptr)))
    return rc;
  pre_back_kernel<<<nblk((int64_t)ns * m), 256, 0, L.st>>>(ns, m, o, d0, Ka, o, C, ns);
  DLAUNCH(L);
  *npn_out = npn;
  return LOBPCG_OK;
}

// svqb (Algorithm 4) / svqbDrop (Algorithm 6) transform, device path.
int svqb_transform_dev(DenseLayer& L, const double* G, int nu, bool drop, double tau, double* T,
                       int* nkeep) {
  DevDense& D = L.dev;
  double* MB = L.A[0];
  double* Z = L.A[3];
  int* est = D.ints + 2;
  int* keep = D.ints + 3;
  int rc;
  dscale2_kernel<<<nblk((int64_t)nu * nu), 256, 0, L.st>>>(nu, G, nu, nullptr, 0, L.d, MB, nullptr,
                                                           nu);
  DLAUNCH(L);
  if ((rc = eig_into(L, nu, MB, Z, est))) return rc;
  svqb_dev_kernel<<<1, 256, 0, L.st>>>(nu, L.ev, L.d, Z, nu, drop ? 1 : 0, tau, T, nu, keep);
  DLAUNCH(L);
  int fl[2];
  if ((rc = read_flags(L, est, 2, nullptr, 0, fl, nullptr))) return rc;
  note_check(L, fl[0]);
  if (fl[0] != 0) {
    if ((rc = eig_recover(L, nu, MB, Z, fl[0]))) return rc;
    svqb_dev_kernel<<<1, 256, 0, L.st>>>(nu, L.ev, L.d, Z, nu, drop ? 1 : 0, tau, T, nu, keep);
    DLAUNCH(L);
    if ((rc = read_flags(L, keep, 1, nullptr, 0, fl + 1, nullptr))) return rc;
  }
  *nkeep = fl[1];
  return LOBPCG_OK;
}

}  // namespace lob
