// Block CSR sparse product Y = A X (the A W, B W products of Algorithm 8 and
// Sec. 5.2), with the diagonal-B product BY = diag(b) X fused into the same
// pass over X.
//
// Layout: X and Y are row-major n x m blocks, so the m values of one row are
// contiguous.  A group of TPR threads (a warp or a power-of-two part of one)
// owns a row: for every nonzero a_ij it reads row j of X with the group's
// lanes on consecutive columns (one coalesced segment per nonzero) and keeps
// the m partial sums in registers.  Stencil neighbours of consecutive rows
// overlap, so neighbour rows are served from L2 and X streams from HBM about
// once.
#include "kernels.cuh"

namespace lob {

int64_t g_launches = 0;

template <int TPR, int CPT>
__global__ void __launch_bounds__(256) spmm_csr_kernel(
    int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ val, const double* __restrict__ X, int64_t ldx, int m,
    double* __restrict__ Y, int64_t ldy, const double* __restrict__ b,
    double* __restrict__ BY, int64_t ldby) {
  const int groups = blockDim.x / TPR;
  const int64_t row = (int64_t)blockIdx.x * groups + threadIdx.x / TPR;
  const int lane = threadIdx.x % TPR;
  if (row >= n) return;
  const int lo = rowptr[row], hi = rowptr[row + 1];
  for (int c0 = 0; c0 < m; c0 += TPR * CPT) {
    double acc[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) acc[t] = 0.0;
    for (int p = lo; p < hi; ++p) {
      const double a = __ldg(val + p);
      const double* xr = X + (int64_t)__ldg(col + p) * ldx;
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        const int c = c0 + lane + t * TPR;
        if (c < m) acc[t] = fma(a, __ldg(xr + c), acc[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      const int c = c0 + lane + t * TPR;
      if (c < m) {
        Y[row * ldy + c] = acc[t];
        if (b && BY) BY[row * ldby + c] = b[row] * X[row * ldx + c];
      }
    }
  }
}

// Wide blocks (m > 32, 16-byte aligned rows): one warp per row; the lanes
// load up to 32 (column, value) pairs of the row at once and broadcast them by
// shuffles, and each lane owns CP column pairs read as double2, so the 8 X
// rows of an unrolled group are in flight together instead of one dependent
// load chain per nonzero.
template <int CP>
__global__ void __launch_bounds__(256) spmm_csr_wide_kernel(
    int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ val, const double* __restrict__ X, int64_t ldx, int m,
    double* __restrict__ Y, int64_t ldy, const double* __restrict__ b,
    double* __restrict__ BY, int64_t ldby) {
  const int64_t row = (int64_t)blockIdx.x * 8 + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= n) return;
  const int lo = rowptr[row], hi = rowptr[row + 1];
  const int npair = (m + 1) / 2;
  double2 acc[CP];
#pragma unroll
  for (int t = 0; t < CP; ++t) acc[t] = make_double2(0.0, 0.0);
  for (int base = lo; base < hi; base += 32) {
    const int cnt = min(32, hi - base);
    const int my_c = lane < cnt ? __ldg(col + base + lane) : 0;
    const double my_v = lane < cnt ? __ldg(val + base + lane) : 0.0;
#pragma unroll 8
    for (int j = 0; j < cnt; ++j) {
      const int c = __shfl_sync(0xffffffffu, my_c, j);
      const double a = __shfl_sync(0xffffffffu, my_v, j);
      const double2* xr = reinterpret_cast<const double2*>(X + (int64_t)c * ldx);
#pragma unroll
      for (int t = 0; t < CP; ++t) {
        const int q = lane + 32 * t;
        if (q < npair) {
          const double2 x = __ldg(xr + q);
          acc[t].x = fma(a, x.x, acc[t].x);
          acc[t].y = fma(a, x.y, acc[t].y);
        }
      }
    }
  }
  const bool fuse = b != nullptr && BY != nullptr;
  const double br = fuse ? b[row] : 0.0;
#pragma unroll
  for (int t = 0; t < CP; ++t) {
    const int q = lane + 32 * t;
    if (q < npair) {
      const int c = 2 * q;
      Y[row * ldy + c] = acc[t].x;
      if (c + 1 < m) Y[row * ldy + c + 1] = acc[t].y;
      if (fuse) {
        const double2 x = __ldg(reinterpret_cast<const double2*>(X + row * ldx) + q);
        BY[row * ldby + c] = br * x.x;
        if (c + 1 < m) BY[row * ldby + c + 1] = br * x.y;
      }
    }
  }
}

template <int CP>
static int launch_spmm_wide(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* col,
                            const double* val, const double* X, int64_t ldx, int m, double* Y,
                            int64_t ldy, const double* b, double* BY, int64_t ldby) {
  spmm_csr_wide_kernel<CP><<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(n, rowptr, col, val, X, ldx,
                                                                     m, Y, ldy, b, BY, ldby);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

template <int TPR, int CPT>
static int launch_spmm(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* col,
                       const double* val, const double* X, int64_t ldx, int m, double* Y,
                       int64_t ldy, const double* b, double* BY, int64_t ldby) {
  const int threads = 256;
  const int64_t rows_per_block = threads / TPR;
  const int64_t blocks = ceil_div(n, rows_per_block);
  spmm_csr_kernel<TPR, CPT><<<(unsigned)blocks, threads, 0, st>>>(n, rowptr, col, val, X, ldx,
                                                                  m, Y, ldy, b, BY, ldby);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

int spmm(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* col,
         const double* val, const double* X, int64_t ldx, int m, double* Y, int64_t ldy,
         const double* b, double* BY, int64_t ldby) {
  if (n <= 0 || m <= 0) return LOBPCG_OK;
  if (m <= 4) return launch_spmm<4, 1>(st, n, rowptr, col, val, X, ldx, m, Y, ldy, b, BY, ldby);
  if (m <= 8) return launch_spmm<8, 1>(st, n, rowptr, col, val, X, ldx, m, Y, ldy, b, BY, ldby);
  if (m <= 16) return launch_spmm<16, 1>(st, n, rowptr, col, val, X, ldx, m, Y, ldy, b, BY, ldby);
  if (m <= 32) return launch_spmm<32, 1>(st, n, rowptr, col, val, X, ldx, m, Y, ldy, b, BY, ldby);
  // double2 path: X rows 16-byte aligned (base and leading dimension even),
  // and an odd m only with a padded row (the pair's second half stays inside it)
  const bool al = ((uintptr_t)X % 16 == 0) && (ldx % 2 == 0) && (m % 2 == 0 || ldx > m);
  if (al && m <= 128)
    return launch_spmm_wide<2>(st, n, rowptr, col, val, X, ldx, m, Y, ldy, b, BY, ldby);
  if (al && m <= 256)
    return launch_spmm_wide<4>(st, n, rowptr, col, val, X, ldx, m, Y, ldy, b, BY, ldby);
  if (m <= 64) return launch_spmm<32, 2>(st, n, rowptr, col, val, X, ldx, m, Y, ldy, b, BY, ldby);
  return launch_spmm<32, 4>(st, n, rowptr, col, val, X, ldx, m, Y, ldy, b, BY, ldby);
}

}  // namespace lob

LOBPCG_EXPORT int lobpcg_spmm(int64_t n, const int32_t* rowptr, const int32_t* col,
                              const double* val, const double* X, int64_t ldx, int64_t m,
                              double* Y, int64_t ldy, const double* b, double* BY,
                              int64_t ldby, void* stream) {
  if (n < 0 || m < 0 || m > (1 << 20)) return LOBPCG_ERR_ARG;
  if (n > 0 && m > 0 && (!rowptr || !col || !val || !X || !Y || ldx < m || ldy < m))
    return LOBPCG_ERR_ARG;
  if (b && (!BY || ldby < m)) return LOBPCG_ERR_ARG;
  if (BY && !b) return LOBPCG_ERR_ARG;
  return lob::spmm((cudaStream_t)stream, n, rowptr, col, val, X, ldx, (int)m, Y, ldy, b, BY,
                   ldby);
}
