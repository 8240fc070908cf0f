// FP64 reference contractions and the fused elementwise passes of one
// iteration of Algorithm 8.
//
//   gram_f64    G = U^T V (block inner products, Sec. 5.2 / Eq. 12-14): the
//               contraction over the n rows is split into row slabs, one CTA
//               per (output tile, slab); the slab partials are summed in a
//               fixed order by a second pass, so results are deterministic.
//   update_f64  Y = beta Y0 + alpha S C (Eq. 10-11): row tiles of S are
//               staged in shared memory and multiplied by C.
//   residual    r_j = AX_j - theta_j BX_j, W = K^-1 R (Jacobi) and the column
//               norms of Eq. (9), one pass over X, AX, BX.
// These run on the FP64 units; the tensor-core versions are in ozaki.cu.
#include <algorithm>

#include "kernels.cuh"

namespace lob {

// ---------------------------------------------------------------- Gram (FP64)

constexpr int kGT = 64;  // output tile
constexpr int kGK = 16;  // rows per shared-memory stage

static void gram_f64_plan(int64_t n, int p, int q, int* slabs, int64_t* rows_per_slab) {
  const int64_t tiles = ceil_div(p, kGT) * ceil_div(q, kGT);
  int64_t s = std::max<int64_t>(1, ceil_div(4 * 152, tiles));
  s = std::min<int64_t>(s, std::max<int64_t>(1, ceil_div(n, 256)));
  int64_t r = round_up(ceil_div(n, s), kGK);
  s = std::max<int64_t>(1, ceil_div(n, r));
  *slabs = (int)s;
  *rows_per_slab = r;
}

int64_t gram_f64_workspace(int64_t n, int p, int q) {
  int slabs;
  int64_t r;
  gram_f64_plan(n, p, q, &slabs, &r);
  return (int64_t)slabs * p * q * (int64_t)sizeof(double);
}

__global__ void __launch_bounds__(256) gram_f64_kernel(int64_t n, SegList U, int p, SegList V,
                                                       int q, int64_t rows_per_slab,
                                                       double* __restrict__ partial) {
  __shared__ double Us[kGK][kGT + 1];
  __shared__ double Vs[kGK][kGT + 1];
  const int tp = blockIdx.x * kGT, tq = blockIdx.y * kGT;
  const int64_t r0 = (int64_t)blockIdx.z * rows_per_slab;
  const int64_t r1 = min(n, r0 + rows_per_slab);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int64_t r = r0; r < r1; r += kGK) {
    for (int e = threadIdx.x; e < kGK * kGT; e += blockDim.x) {
      const int rr = e / kGT, cc = e % kGT;
      const int64_t row = r + rr;
      const bool ok = row < r1;
      Us[rr][cc] = (ok && tp + cc < p) ? seg_load(U, tp + cc, row) : 0.0;
      Vs[rr][cc] = (ok && tq + cc < q) ? seg_load(V, tq + cc, row) : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kGK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Us[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Vs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* out = partial + (int64_t)blockIdx.z * p * q;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gi = tp + ty + 16 * i, gj = tq + tx + 16 * j;
      if (gi < p && gj < q) out[(int64_t)gi * q + gj] = acc[i][j];
    }
}

__global__ void slab_reduce_kernel(const double* __restrict__ partial, int slabs, int p, int q,
                                   double* __restrict__ G, int64_t ldg) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)p * q) return;
  double s = 0.0;
  for (int z = 0; z < slabs; ++z) s += partial[(int64_t)z * p * q + e];
  const int i = (int)(e / q), j = (int)(e % q);
  G[i + (int64_t)j * ldg] = s;
}

int gram_f64(cudaStream_t st, int64_t n, const SegList& U, const SegList& V, double* G,
             int64_t ldg, void* work, int64_t work_bytes) {
  const int p = U.off[U.nseg], q = V.off[V.nseg];
  if (p <= 0 || q <= 0) return LOBPCG_OK;
  int slabs;
  int64_t rps;
  gram_f64_plan(std::max<int64_t>(n, 1), p, q, &slabs, &rps);
  if (work_bytes < (int64_t)slabs * p * q * (int64_t)sizeof(double)) return LOBPCG_ERR_ARG;
  double* partial = (double*)work;
  if (n > 0) {
    dim3 grid((unsigned)ceil_div(p, kGT), (unsigned)ceil_div(q, kGT), (unsigned)slabs);
    gram_f64_kernel<<<grid, 256, 0, st>>>(n, U, p, V, q, rps, partial);
    LOB_LAUNCHED();
  } else {
    slabs = 1;
    LOB_CUDA_OK(cudaMemsetAsync(partial, 0, (size_t)p * q * sizeof(double), st));
  }
  const int64_t tot = (int64_t)p * q;
  slab_reduce_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(partial, slabs, p, q, G, ldg);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

// -------------------------------------------------------------- update (FP64)

constexpr int kUT = 64;  // rows and output columns per tile
constexpr int kUK = 16;  // contraction stage

__global__ void __launch_bounds__(256) update_f64_kernel(int64_t n, SegList S, int s,
                                                         const double* __restrict__ C,
                                                         int64_t ldc, int m, double alpha,
                                                         double beta, SegList Y0, OutList Y) {
  __shared__ double Ss[kUT][kUK + 1];
  __shared__ double Cs[kUK][kUT + 1];
  const int64_t r0 = (int64_t)blockIdx.x * kUT;
  const int c0 = blockIdx.y * kUT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < s; k0 += kUK) {
    for (int e = threadIdx.x; e < kUT * kUK; e += blockDim.x) {
      const int rr = e / kUK, kk = e % kUK;
      const int64_t row = r0 + rr;
      Ss[rr][kk] = (row < n && k0 + kk < s) ? seg_load(S, k0 + kk, row) : 0.0;
      const int kc = e / kUT, cc = e % kUT;
      Cs[kc][cc] = (k0 + kc < s && c0 + cc < m) ? C[(k0 + kc) + (int64_t)(c0 + cc) * ldc] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kUK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ss[ty + 16 * i][k];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Cs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t row = r0 + ty + 16 * i;
      const int c = c0 + tx + 16 * j;
      if (row < n && c < m) {
        double v = alpha * acc[i][j];
        if (beta != 0.0) v = fma(beta, seg_load(Y0, c, row), v);
        *out_addr(Y, c, row) = v;
      }
    }
}

int update_f64(cudaStream_t st, int64_t n, const SegList& S, const double* C, int64_t ldc,
               int m, double alpha, double beta, const SegList& Y0, const OutList& Y) {
  const int s = S.off[S.nseg];
  if (n <= 0 || m <= 0) return LOBPCG_OK;
  dim3 grid((unsigned)ceil_div(n, kUT), (unsigned)ceil_div(m, kUT));
  update_f64_kernel<<<grid, 256, 0, st>>>(n, S, s, C, ldc, m, alpha, beta, Y0, Y);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

// ------------------------------------------------------- residual and norms

// kinv = 1 / kdiag: the preconditioner is applied as a product, because an
// FP64 division costs ~10 FP64 instructions on a part whose FP64 rate is 1/64
// of FP32 (the residual pass was bound by it)
__global__ void reciprocal_kernel(int64_t n, const double* __restrict__ d,
                                  double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = 1.0 / d[i];
}

int reciprocal(cudaStream_t st, int64_t n, const double* d, double* out) {
  if (n <= 0) return LOBPCG_OK;
  reciprocal_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(n, d, out);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

static int row_blocks(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 64), 4 * 152));
}

int64_t residual_workspace(int64_t n, int m) {
  return (int64_t)row_blocks(n) * 2 * std::max(m, 1) * (int64_t)sizeof(double);
}

// Block: 32 columns x 8 row lanes; each block owns a contiguous row range.
__global__ void __launch_bounds__(256) residual_kernel(
    int64_t n, const double* __restrict__ X, const double* __restrict__ AX,
    const double* __restrict__ BX, int64_t ld, int m, int c0, const double* __restrict__ theta,
    const double* __restrict__ kinv, double* __restrict__ W, int64_t ldw, int xb,
    double* __restrict__ partial) {
  __shared__ double red[2][8][33];
  const int mm = m - c0;
  const int64_t per = ceil_div(n, (int64_t)gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(n, r0 + per);
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int cb = 0; cb < mm; cb += 32) {
    const int j = c0 + cb + tx;
    double rn = 0.0, xn = 0.0;
    if (j < m) {
      const double th = theta[j];
#pragma unroll 4
      for (int64_t r = r0 + ty; r < r1; r += 8) {
        const int64_t o = r * ld + j;
        const double x = X[o];
        const double bx = BX ? BX[o] : x;
        const double res = fma(-th, bx, AX[o]);
        rn = fma(res, res, rn);
        xn = fma(x, xb ? bx : x, xn);  // ||x||^2, or x^T B x for criterion (8)
        if (W) W[r * ldw + (j - c0)] = kinv ? res * kinv[r] : res;
      }
    }
    red[0][ty][tx] = rn;
    red[1][ty][tx] = xn;
    __syncthreads();
    if (ty == 0 && j < m) {
      double a = 0.0, b = 0.0;
      for (int t = 0; t < 8; ++t) {
        a += red[0][t][tx];
        b += red[1][t][tx];
      }
      partial[((int64_t)blockIdx.x * 2 + 0) * mm + (j - c0)] = a;
      partial[((int64_t)blockIdx.x * 2 + 1) * mm + (j - c0)] = b;
    }
    __syncthreads();
  }
}

__global__ void residual_finish_kernel(const double* __restrict__ partial, int blocks, int mm,
                                       int c0, const double* __restrict__ theta, double normA,
                                       double normB, double* __restrict__ be) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= mm) return;
  double a = 0.0, b = 0.0;
  for (int z = 0; z < blocks; ++z) {
    a += partial[((int64_t)z * 2 + 0) * mm + j];
    b += partial[((int64_t)z * 2 + 1) * mm + j];
  }
  be[j] = sqrt(a) / ((normA + fabs(theta[c0 + j]) * normB) * sqrt(b));
}

int residual(cudaStream_t st, int64_t n, const double* X, const double* AX, const double* BX,
             int64_t ld, int m, int c0, const double* theta, const double* kinv, double* W,
             int64_t ldw, double normA, double normB, double* be, void* partial, int xb) {
  const int mm = m - c0;
  if (mm <= 0) return LOBPCG_OK;
  const int blocks = row_blocks(n);
  residual_kernel<<<blocks, 256, 0, st>>>(n, X, AX, BX, ld, m, c0, theta, kinv, W, ldw, xb,
                                          (double*)partial);
  LOB_LAUNCHED();
  residual_finish_kernel<<<(unsigned)ceil_div(mm, 128), 128, 0, st>>>(
      (const double*)partial, blocks, mm, c0, theta, normA, normB, be);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

// ------------------------------------------------------- column sums of squares

int64_t colsumsq_workspace(int64_t n, int m) {
  return (int64_t)row_blocks(n) * std::max(m, 1) * (int64_t)sizeof(double);
}

__global__ void __launch_bounds__(256) colsumsq_kernel(int64_t n, const double* __restrict__ Y,
                                                       int64_t ld, int m,
                                                       double* __restrict__ partial) {
  __shared__ double red[8][33];
  const int64_t per = ceil_div(n, (int64_t)gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(n, r0 + per);
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int cb = 0; cb < m; cb += 32) {
    const int j = cb + tx;
    double s = 0.0;
    if (j < m)
      for (int64_t r = r0 + ty; r < r1; r += 8) {
        const double y = Y[r * ld + j];
        s = fma(y, y, s);
      }
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && j < m) {
      double a = 0.0;
      for (int t = 0; t < 8; ++t) a += red[t][tx];
      partial[(int64_t)blockIdx.x * m + j] = a;
    }
    __syncthreads();
  }
}

__global__ void colsum_finish_kernel(const double* __restrict__ partial, int blocks, int m,
                                     double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double a = 0.0;
  for (int z = 0; z < blocks; ++z) a += partial[(int64_t)z * m + j];
  out[j] = a;
}

int colsumsq(cudaStream_t st, int64_t n, const double* Y, int64_t ld, int m, double* out,
             void* partial) {
  if (m <= 0) return LOBPCG_OK;
  const int blocks = row_blocks(n);
  colsumsq_kernel<<<blocks, 256, 0, st>>>(n, Y, ld, m, (double*)partial);
  LOB_LAUNCHED();
  colsum_finish_kernel<<<(unsigned)ceil_div(m, 128), 128, 0, st>>>((const double*)partial,
                                                                   blocks, m, out);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

// ------------------------------------------------------------- elementwise

__global__ void diag_scale_kernel(int64_t n, int m, const double* __restrict__ b,
                                  const double* __restrict__ X, int64_t ldx,
                                  double* __restrict__ Y, int64_t ldy) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  const int64_t r = e / m;
  const int c = (int)(e % m);
  Y[r * ldy + c] = b[r] * X[r * ldx + c];
}

int diag_scale(cudaStream_t st, int64_t n, int m, const double* b, const double* X,
               int64_t ldx, double* Y, int64_t ldy) {
  if (n <= 0 || m <= 0) return LOBPCG_OK;
  diag_scale_kernel<<<(unsigned)ceil_div(n * m, 256), 256, 0, st>>>(n, m, b, X, ldx, Y, ldy);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

__global__ void copy_block_kernel(int64_t n, int m, const double* __restrict__ X, int64_t ldx,
                                  double* __restrict__ Y, int64_t ldy) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  const int64_t r = e / m;
  const int c = (int)(e % m);
  Y[r * ldy + c] = X[r * ldx + c];
}

int copy_block(cudaStream_t st, int64_t n, int m, const double* X, int64_t ldx, double* Y,
               int64_t ldy) {
  if (n <= 0 || m <= 0) return LOBPCG_OK;
  copy_block_kernel<<<(unsigned)ceil_div(n * m, 256), 256, 0, st>>>(n, m, X, ldx, Y, ldy);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

// One block per column: find the largest |x| (lowest row on ties), flip the sign.
__global__ void __launch_bounds__(256) sign_normalise_kernel(int64_t n, double* X, int64_t ldx) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  const int j = blockIdx.x;
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double a = fabs(X[r * ldx + j]);
    if (a > best) {
      best = a;
      bi = r;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sv[threadIdx.x + s];
      const int64_t oi = si[threadIdx.x + s];
      if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  // decide once: a thread that flips its rows must not change the value the
  // others read
  __shared__ int flip_s;
  if (threadIdx.x == 0) flip_s = X[si[0] * ldx + j] < 0.0 ? 1 : 0;
  __syncthreads();
  const bool flip = flip_s != 0;
  if (flip)
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) X[r * ldx + j] = -X[r * ldx + j];
}

int64_t sign_normalise_workspace(int64_t, int) { return 0; }

int sign_normalise(cudaStream_t st, int64_t n, int m, double* X, int64_t ldx, void*) {
  if (n <= 0 || m <= 0) return LOBPCG_OK;
  sign_normalise_kernel<<<m, 256, 0, st>>>(n, X, ldx);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

// ------------------------------------------------------ balance exponents
// out[k] = floor(log2(G_kk) / 2), i.e. 2^out[k] is within a factor 2 of the
// column norm sqrt(G_kk) (0 for a non-positive diagonal).  Integer ops only.
__global__ void diag_exponents_kernel(int n, const double* __restrict__ G, int64_t ldg,
                                      int* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const long long b = __double_as_longlong(G[k + (int64_t)k * ldg]);
  const int be = (int)((b >> 52) & 0x7FF);
  int e = 0;
  if (b > 0 && be > 0 && be < 0x7FF) {
    const int u = be - 1023;
    e = (u >= 0) ? u / 2 : -((-u + 1) / 2);
  }
  out[k] = e;
}

int diag_exponents(cudaStream_t st, int n, const double* G, int64_t ldg, int* out) {
  if (n <= 0) return LOBPCG_OK;
  diag_exponents_kernel<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(n, G, ldg, out);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

// ------------------------------------------------------------- Philox4x32-10
// Salmon et al. (SC'11): ten rounds of two 32x32->64 multiplications with the
// constants 0xD2511F53 / 0xCD9E8D57 and a Weyl key schedule 0x9E3779B9 /
// 0xBB67AE85.

__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ double uniform52(uint32_t a, uint32_t b) {
  const uint64_t m = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
  return ((double)m + 0.5) * 0x1p-52;
}

__global__ void philox_normal_kernel(int64_t total, int m, uint32_t k0, uint32_t k1,
                                     uint32_t sid, double* __restrict__ Y, int64_t ldy) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t f0 = 2 * j;
  if (f0 >= total) return;
  const uint4 o = philox10(make_uint4((uint32_t)j, (uint32_t)((uint64_t)j >> 32), sid, 0u), k0, k1);
  const double u1 = uniform52(o.x, o.y), u2 = uniform52(o.z, o.w);
  const double rad = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  Y[(f0 / m) * ldy + (f0 % m)] = rad * cs;
  if (f0 + 1 < total) Y[((f0 + 1) / m) * ldy + ((f0 + 1) % m)] = rad * sn;
}

int philox_normal(cudaStream_t st, int64_t n, int m, uint64_t seed, uint32_t stream_id,
                  double* Y, int64_t ldy) {
  const int64_t total = n * m;
  if (total <= 0) return LOBPCG_OK;
  const int64_t pairs = ceil_div(total, 2);
  philox_normal_kernel<<<(unsigned)ceil_div(pairs, 256), 256, 0, st>>>(
      total, m, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), stream_id, Y, ldy);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

}  // namespace lob

// ------------------------------------------------------------ C ABI wrappers

static bool seg_ok(const double* p, int64_t ld, int64_t cols) { return p && ld >= cols; }

LOBPCG_EXPORT int64_t lobpcg_gram_workspace(int64_t n, int64_t p, int64_t q, int mode,
                                            int slices) {
  if (n < 0 || p < 0 || q < 0) return -1;
  if (mode == LOBPCG_GEMM_OZAKI) return lob::gram_ozaki_workspace(n, (int)p, (int)q, slices);
  if (mode == LOBPCG_GEMM_OZAKI_TC)
    return std::max(lob::gram_tc_workspace(n, (int)p, (int)q),
                    lob::gram_ozaki_workspace(n, (int)p, (int)q, slices));
  return lob::gram_f64_workspace(n, (int)p, (int)q);
}

LOBPCG_EXPORT int lobpcg_gram(int64_t n, const double* U, int64_t ldu, int64_t p,
                              const double* V, int64_t ldv, int64_t q, double* G, int64_t ldg,
                              int mode, int slices, void* work, int64_t work_bytes,
                              void* stream) {
  if (n < 0 || p < 0 || q < 0 || p > (1 << 20) || q > (1 << 20)) return LOBPCG_ERR_ARG;
  if (p == 0 || q == 0) return LOBPCG_OK;
  if (!G || ldg < p || (n > 0 && (!seg_ok(U, ldu, p) || !seg_ok(V, ldv, q))))
    return LOBPCG_ERR_ARG;
  if (mode != LOBPCG_GEMM_F64 && mode != LOBPCG_GEMM_OZAKI && mode != LOBPCG_GEMM_OZAKI_TC)
    return LOBPCG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t need = lobpcg_gram_workspace(n, p, q, mode, slices);
  void* own = nullptr;
  if (!work) {
    if (cudaMallocAsync(&own, (size_t)std::max<int64_t>(need, 16), st) != cudaSuccess)
      return LOBPCG_ERR_OOM;
    work = own;
    work_bytes = need;
  }
  lob::SegList Us = lob::seg1(U, ldu, (int)p), Vs = lob::seg1(V, ldv, (int)q);
  int rc = mode == LOBPCG_GEMM_OZAKI_TC
               ? lob::gram_tc(st, n, Us, Vs, G, ldg, slices, work, work_bytes)
               : mode == LOBPCG_GEMM_OZAKI
                     ? lob::gram_ozaki(st, n, Us, Vs, G, ldg, slices, work, work_bytes)
                     : lob::gram_f64(st, n, Us, Vs, G, ldg, work, work_bytes);
  if (own) cudaFreeAsync(own, st);
  return rc;
}

LOBPCG_EXPORT int lobpcg_wait_selftest(int32_t polls, void* stream) {
  if (polls < 1) return LOBPCG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return LOBPCG_ERR_OOM;
  int h = 0;
  bool ok = cudaMemsetAsync(d, 0, sizeof(int), st) == cudaSuccess &&
            lob::wait_selftest(st, polls, d) == LOBPCG_OK &&
            cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(d);
  if (!ok) return LOBPCG_ERR_CUDA;
  return (h & 1) ? LOBPCG_ERR_TIMEOUT : LOBPCG_OK;
}

LOBPCG_EXPORT int lobpcg_update(int64_t n, const double* S, int64_t lds, int64_t s,
                                const double* C, int64_t ldc, int64_t m, double alpha,
                                double beta, const double* Y0, int64_t ldy0, double* Y,
                                int64_t ldy, int mode, int slices, void* stream) {
  if (n < 0 || s < 0 || m < 0 || s > (1 << 20) || m > (1 << 20)) return LOBPCG_ERR_ARG;
  if (n == 0 || m == 0) return LOBPCG_OK;
  if (!Y || ldy < m || (s > 0 && (!seg_ok(S, lds, s) || !C || ldc < s))) return LOBPCG_ERR_ARG;
  if (beta != 0.0 && !seg_ok(Y0, ldy0, m)) return LOBPCG_ERR_ARG;
  if (mode != LOBPCG_GEMM_F64 && mode != LOBPCG_GEMM_OZAKI && mode != LOBPCG_GEMM_OZAKI_TC)
    return LOBPCG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  lob::SegList Ss = s > 0 ? lob::seg1(S, lds, (int)s) : lob::seg_empty();
  lob::SegList Y0s = beta != 0.0 ? lob::seg1(Y0, ldy0, (int)m) : lob::seg_empty();
  lob::OutList out{{Y, Y}, {ldy, ldy}, (int)m};
  if (mode == LOBPCG_GEMM_OZAKI || mode == LOBPCG_GEMM_OZAKI_TC) {
    const bool tc = mode == LOBPCG_GEMM_OZAKI_TC;
    const int64_t need = tc ? lob::update_tc_workspace(n, (int)s, (int)m, slices)
                            : lob::update_ozaki_workspace(n, (int)s, (int)m, slices);
    void* own = nullptr;
    if (need > 0 && cudaMallocAsync(&own, (size_t)need, st) != cudaSuccess) return LOBPCG_ERR_OOM;
    int rc = tc ? lob::update_tc(st, n, Ss, C, ldc, (int)m, alpha, beta, Y0s, out, slices, own,
                                 need)
                : lob::update_ozaki(st, n, Ss, C, ldc, (int)m, alpha, beta, Y0s, out, slices,
                                    own, need);
    if (own) cudaFreeAsync(own, st);
    return rc;
  }
  return lob::update_f64(st, n, Ss, C, ldc, (int)m, alpha, beta, Y0s, out);
}

LOBPCG_EXPORT int lobpcg_residual(int64_t n, const double* X, const double* AX,
                                  const double* BX, int64_t ld, int64_t m, int64_t c0,
                                  const double* theta, const double* kdiag, double* W,
                                  int64_t ldw, double normA, double normB, double* be,
                                  void* stream) {
  if (n <= 0 || m < 0 || c0 < 0 || c0 > m || m > (1 << 20)) return LOBPCG_ERR_ARG;
  if (c0 == m) return LOBPCG_OK;
  if (!X || !AX || ld < m || !theta || !be || (W && ldw < m - c0)) return LOBPCG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  void* part = nullptr;
  const size_t pb = (size_t)lob::residual_workspace(n, (int)(m - c0));
  if (cudaMallocAsync(&part, pb + (kdiag ? (size_t)n * sizeof(double) : 0), st) != cudaSuccess)
    return LOBPCG_ERR_OOM;
  double* kinv = kdiag ? (double*)((char*)part + pb) : nullptr;
  int rc = kdiag ? lob::reciprocal(st, n, kdiag, kinv) : LOBPCG_OK;
  if (!rc)
    rc = lob::residual(st, n, X, AX, BX, ld, (int)m, (int)c0, theta, kinv, W, ldw, normA, normB,
                       be, part);
  cudaFreeAsync(part, st);
  return rc;
}

LOBPCG_EXPORT int lobpcg_philox_normal(int64_t n, int64_t m, uint64_t seed, uint32_t stream_id,
                                       double* Y, int64_t ldy, void* stream) {
  if (n < 0 || m < 0 || (n > 0 && m > 0 && (!Y || ldy < m))) return LOBPCG_ERR_ARG;
  return lob::philox_normal((cudaStream_t)stream, n, (int)m, seed, stream_id, Y, ldy);
}
