// Adjoint kernels of the eigenpair gradients (not in the paper: first-order
// perturbation theory of the pencil A x = lambda B x with B-orthonormal x).
//
// For upstream gradients gl_i = dL/dlambda_i and g_i = dL/dx_i of the k
// wanted pairs,
//   w_i = sum_{j != i} x_j (x_j^T g_i) / (lambda_i - lambda_j) = w_i^in - u_i,
// w_i^in over the k known pairs, u_i the solution on the B-orthogonal
// complement of X of (A - lambda_i B) u_i = (I - B X X^T) g_i, found by a
// projected, Jacobi-preconditioned conjugate gradient per column (the shifted
// operator is positive definite there when lambda_{k+1} > lambda_k).  Then
//   dL/dA = sum_i gl_i x_i x_i^T + sym(w_i x_i^T)
//   dL/dB = sum_i -lambda_i gl_i x_i x_i^T - lambda_i sym(w_i x_i^T)
//                 - 1/2 (g_i^T x_i) x_i x_i^T
// sampled on the CSR patterns of A and B (or the diagonal of a diagonal B).
//
// GB300 mapping: every n-scaled step streams row-major n x k blocks once
// (coalesced across the k columns of a row); column dot products are two-pass
// fixed-order reductions (deterministic); the per-column CG scalars are read
// from device memory by the kernels that use them, so a CG iteration needs no
// host round trip.
#include <algorithm>

#include "kernels.cuh"

namespace lob {
namespace {

constexpr int kRB = 152 * 4;  // row blocks of the column reductions

__device__ __forceinline__ double safe_div(double a, double b) {
  return (b != 0.0 && isfinite(a / b)) ? a / b : 0.0;
}

// Cin(j, i) = M(j, i) / (lambda_i - lambda_j), j != i (column-major k x k);
// flag = 1 when a pair is closer than gap (absolute).
__global__ void adj_coeff_kernel(int k, const double* __restrict__ M, int64_t ldm,
                                 const double* __restrict__ lam, double gap,
                                 double* __restrict__ Cin, int* __restrict__ flag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * k) return;
  const int j = (int)(e % k), i = (int)(e / k);
  double c = 0.0;
  if (i != j) {
    const double d = lam[i] - lam[j];
    if (!(fabs(d) >= gap)) atomicExch(flag, 1);
    c = fabs(d) > 0.0 ? M[j + (int64_t)i * ldm] / d : 0.0;
  }
  Cin[j + (int64_t)i * k] = c;
}

// Block-local column sums of the per-thread partials s (8 warps x 32 columns)
// into partial[blockIdx.x * k + j].
__device__ __forceinline__ void block_colsum(double s, int j, int k, double (*red)[33],
                                             double* __restrict__ partial) {
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  red[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && j < k) {
    double a = 0.0;
    for (int t = 0; t < 8; ++t) a += red[t][tx];
    partial[(int64_t)blockIdx.x * k + j] = a;
  }
  __syncthreads();
}

// Q(r, j) -= lambda_j * (B P)(r, j) and partial column dots P(:, j)^T Q(:, j).
// (B P) is BP when given, b[r] P(r, j) for a diagonal B, else P.
__global__ void __launch_bounds__(256) shift_dot_kernel(
    int64_t n, int k, double* __restrict__ Q, const double* __restrict__ P,
    const double* __restrict__ BP, const double* __restrict__ b, int64_t ld,
    const double* __restrict__ lam, double* __restrict__ partial) {
  __shared__ double red[8][33];
  const int64_t per = ceil_div(n, (int64_t)gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(n, r0 + per);
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int cb = 0; cb < k; cb += 32) {
    const int j = cb + tx;
    double s = 0.0;
    if (j < k) {
      const double l = lam[j];
      for (int64_t r = r0 + ty; r < r1; r += 8) {
        const int64_t o = r * ld + j;
        const double p = P[o];
        const double bp = BP ? BP[o] : (b ? b[r] * p : p);
        const double q = fma(-l, bp, Q[o]);
        Q[o] = q;
        s = fma(p, q, s);
      }
    }
    block_colsum(s, j, k, red, partial);
  }
}

// CG step with alpha_j = rz_j / pq_j (0 for a finished or broken column):
// V -= alpha P (V accumulates -u), R -= alpha Q, Z = R kinv (kinv = 1 / diag
// of the preconditioner), partial R^T R.
// V may alias P and R may alias Q (the first step runs with alpha = 0 on
// V = P = 0, R = Q = F to form Z = K^-1 F and |F|^2).
__global__ void __launch_bounds__(256) cg_step_kernel(
    int64_t n, int k, double* V, const double* P, double* R, const double* Q,
    double* __restrict__ Z, const double* __restrict__ kinv, int64_t ld,
    const double* __restrict__ rz, const double* __restrict__ pq, double* __restrict__ partial) {
  __shared__ double red[8][33];
  const int64_t per = ceil_div(n, (int64_t)gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(n, r0 + per);
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int cb = 0; cb < k; cb += 32) {
    const int j = cb + tx;
    double s = 0.0;
    if (j < k) {
      const double a = pq[j] > 0.0 ? safe_div(rz[j], pq[j]) : 0.0;
      for (int64_t r = r0 + ty; r < r1; r += 8) {
        const int64_t o = r * ld + j;
        V[o] = fma(-a, P[o], V[o]);
        const double rr = fma(-a, Q[o], R[o]);
        R[o] = rr;
        Z[o] = kinv ? rr * kinv[r] : rr;
        s = fma(rr, rr, s);
      }
    }
    block_colsum(s, j, k, red, partial);
  }
}

// partial column dots X(:, j)^T Y(:, j)
__global__ void __launch_bounds__(256) coldot_kernel(int64_t n, int k,
                                                     const double* __restrict__ X,
                                                     const double* __restrict__ Y, int64_t ld,
                                                     double* __restrict__ partial) {
  __shared__ double red[8][33];
  const int64_t per = ceil_div(n, (int64_t)gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(n, r0 + per);
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int cb = 0; cb < k; cb += 32) {
    const int j = cb + tx;
    double s = 0.0;
    if (j < k)
      for (int64_t r = r0 + ty; r < r1; r += 8) s = fma(X[r * ld + j], Y[r * ld + j], s);
    block_colsum(s, j, k, red, partial);
  }
}

__global__ void colfinish_kernel(const double* __restrict__ partial, int blocks, int k,
                                 double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double a = 0.0;
  for (int z = 0; z < blocks; ++z) a += partial[(int64_t)z * k + j];
  out[j] = a;
}

// P = Z + beta P, beta_j = rz_new_j / rz_old_j (0 when rz_old_j == 0)
__global__ void cg_direction_kernel(int64_t n, int k, double* __restrict__ P,
                                    const double* __restrict__ Z, int64_t ld,
                                    const double* __restrict__ rz_new,
                                    const double* __restrict__ rz_old) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int64_t r = e / k;
  const int j = (int)(e % k);
  const double beta = rz_old[j] > 0.0 ? safe_div(rz_new[j], rz_old[j]) : 0.0;
  const int64_t o = r * ld + j;
  P[o] = fma(beta, P[o], Z[o]);
}

// Gradient on a CSR pattern, one warp per row r; for each stored (r, c):
//   out = sum_i ca_i x_ri x_ci + cw_i (w_ri x_ci + x_ri w_ci) / 2
// (ca_i = gl_i, cw_i = 1 for A; ca_i = -lambda_i gl_i - (g_i^T x_i)/2,
// cw_i = -lambda_i for B).
__global__ void __launch_bounds__(256) pattern_grad_kernel(
    int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ X, const double* __restrict__ W, int64_t ld, int k,
    const double* __restrict__ ca, const double* __restrict__ cw, double* __restrict__ out) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (r >= n) return;
  const int32_t e0 = rowptr[r], e1 = rowptr[r + 1];
  for (int32_t e = e0; e < e1; ++e) {
    const int64_t c = col[e];
    double s = 0.0;
    for (int i = lane; i < k; i += 32) {
      const double xr = X[r * ld + i], xc = X[c * ld + i];
      const double wr = W[r * ld + i], wc = W[c * ld + i];
      s = fma(ca[i] * xr, xc, s);
      s = fma(0.5 * cw[i], fma(wr, xc, xr * wc), s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[e] = s;
  }
}

// Diagonal metric: out[r] = sum_i ca_i x_ri^2 + cw_i w_ri x_ri
__global__ void __launch_bounds__(256) diag_grad_kernel(int64_t n, const double* __restrict__ X,
                                                        const double* __restrict__ W, int64_t ld,
                                                        int k, const double* __restrict__ ca,
                                                        const double* __restrict__ cw,
                                                        double* __restrict__ out) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (r >= n) return;
  double s = 0.0;
  for (int i = lane; i < k; i += 32) {
    const double x = X[r * ld + i], w = W[r * ld + i];
    s = fma(ca[i] * x, x, s);
    s = fma(cw[i] * w, x, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[r] = s;
}

// ca/cw coefficients of dL/dA and dL/dB; M = X^T G (column-major, leading
// dimension ldm) gives g_i^T x_i = M(i, i).
__global__ void grad_coeff_kernel(int k, const double* __restrict__ lam,
                                  const double* __restrict__ glam, const double* __restrict__ M,
                                  int64_t ldm, double* __restrict__ caA,
                                  double* __restrict__ cwA, double* __restrict__ caB,
                                  double* __restrict__ cwB) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const double gl = glam ? glam[i] : 0.0;
  const double gx = M ? M[i + (int64_t)i * ldm] : 0.0;
  caA[i] = gl;
  cwA[i] = 1.0;
  caB[i] = -lam[i] * gl - 0.5 * gx;
  cwB[i] = -lam[i];
}

int col_finish(cudaStream_t st, int k, void* partial, double* out) {
  colfinish_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, st>>>((const double*)partial, kRB, k,
                                                               out);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

}  // namespace

int adj_coeff(cudaStream_t st, int k, const double* M, int64_t ldm, const double* lam, double gap,
              double* Cin, int* flag) {
  if (k <= 0) return LOBPCG_OK;
  adj_coeff_kernel<<<(unsigned)ceil_div((int64_t)k * k, 256), 256, 0, st>>>(k, M, ldm, lam, gap,
                                                                            Cin, flag);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

int64_t adj_reduce_workspace(int k) { return (int64_t)kRB * std::max(k, 1) * sizeof(double); }

int shift_dot(cudaStream_t st, int64_t n, int k, double* Q, const double* P, const double* BP,
              const double* b, int64_t ld, const double* lam, double* out, void* partial) {
  shift_dot_kernel<<<kRB, 256, 0, st>>>(n, k, Q, P, BP, b, ld, lam, (double*)partial);
  LOB_LAUNCHED();
  return col_finish(st, k, partial, out);
}

int cg_step(cudaStream_t st, int64_t n, int k, double* V, const double* P, double* R,
            const double* Q, double* Z, const double* kinv, int64_t ld, const double* rz,
            const double* pq, double* rr, void* partial) {
  cg_step_kernel<<<kRB, 256, 0, st>>>(n, k, V, P, R, Q, Z, kinv, ld, rz, pq, (double*)partial);
  LOB_LAUNCHED();
  return col_finish(st, k, partial, rr);
}

int coldot(cudaStream_t st, int64_t n, int k, const double* X, const double* Y, int64_t ld,
           double* out, void* partial) {
  coldot_kernel<<<kRB, 256, 0, st>>>(n, k, X, Y, ld, (double*)partial);
  LOB_LAUNCHED();
  return col_finish(st, k, partial, out);
}

int cg_direction(cudaStream_t st, int64_t n, int k, double* P, const double* Z, int64_t ld,
                 const double* rz_new, const double* rz_old) {
  cg_direction_kernel<<<(unsigned)ceil_div(n * k, 256), 256, 0, st>>>(n, k, P, Z, ld, rz_new,
                                                                      rz_old);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

int grad_coeff(cudaStream_t st, int k, const double* lam, const double* glam, const double* M,
               int64_t ldm, double* caA, double* cwA, double* caB, double* cwB) {
  grad_coeff_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, st>>>(k, lam, glam, M, ldm, caA, cwA,
                                                                caB, cwB);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

int pattern_grad(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* col,
                 const double* X, const double* W, int64_t ld, int k, const double* ca,
                 const double* cw, double* out) {
  pattern_grad_kernel<<<(unsigned)ceil_div(n * 32, 256), 256, 0, st>>>(n, rowptr, col, X, W, ld,
                                                                       k, ca, cw, out);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

int diag_grad(cudaStream_t st, int64_t n, const double* X, const double* W, int64_t ld, int k,
              const double* ca, const double* cw, double* out) {
  diag_grad_kernel<<<(unsigned)ceil_div(n * 32, 256), 256, 0, st>>>(n, X, W, ld, k, ca, cw, out);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

}  // namespace lob
