// Internal launchers of the n-scaled kernels (all device pointers, stream-ordered).
#pragma once
#include "common.cuh"

namespace lob {

// Y = A X (and BY = diag(b) X when b != nullptr); CSR A, X n x m row-major.
int spmm(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* col,
         const double* val, const double* X, int64_t ldx, int m, double* Y, int64_t ldy,
         const double* b, double* BY, int64_t ldby);

// G = U^T V (G column-major, leading dimension ldg), plain FP64 on the CUDA
// cores with a split over rows and a fixed-order second pass (deterministic).
int64_t gram_f64_workspace(int64_t n, int p, int q);
int gram_f64(cudaStream_t st, int64_t n, const SegList& U, const SegList& V, double* G,
             int64_t ldg, void* work, int64_t work_bytes);

// G = U^T V with FP64 emulated through exact BF16 slices on the tensor cores.
int64_t gram_ozaki_workspace(int64_t n, int p, int q, int slices);
int gram_ozaki(cudaStream_t st, int64_t n, const SegList& U, const SegList& V, double* G,
               int64_t ldg, int slices, void* work, int64_t work_bytes);

// Fixed-order sum of Ozaki slab partials (hi, lo, exponent) into G (column-major).
int ozaki_slab_reduce(cudaStream_t st, const float4* partial, int slabs, int p, int q, double* G,
                      int64_t ldg);

// Same Gram on the tcgen05 tensor cores with TMEM accumulators (ozaki_tc.cu).
int64_t gram_tc_workspace(int64_t n, int p, int q);
int gram_tc(cudaStream_t st, int64_t n, const SegList& U, const SegList& V, double* G,
            int64_t ldg, int slices, void* work, int64_t work_bytes);

// Y = beta Y0 + alpha S C on tcgen05 (beta 0 or 1), colexp as update_ozaki.
int64_t update_tc_workspace(int64_t n, int s, int m, int slices);
// status (device int, may be null): bit 0 set when a bounded wait of the
// tensor-core kernel ran out (its outputs are then not valid).
int update_tc(cudaStream_t st, int64_t n, const SegList& S, const double* C, int64_t ldc, int m,
              double alpha, double beta, const SegList& Y0, const OutList& Y, int slices,
              void* work, int64_t work_bytes, const int* colexp = nullptr,
              int* status = nullptr);

// One CTA whose bounded mbarrier wait (at most `limit` polls) on a phase that
// nothing completes must run out: sets bit 0 of *status (device int).
int wait_selftest(cudaStream_t st, int limit, int* status);

// colexp[k] = E with max_i |S(i, k)| < 2^E over an n x s block (0 for zero columns).
int column_exponents(cudaStream_t st, int64_t n, const SegList& Sg, int s, int* out);

// As gram_ozaki, with as many row slabs as fit in work_bytes (fixed scratch).
int gram_ozaki_bounded(cudaStream_t st, int64_t n, const SegList& U, const SegList& V, double* G,
                       int64_t ldg, int slices, void* work, int64_t work_bytes);

// Y = beta * Y0 + alpha * S C; S segments (n x s), C s x m column-major.
int update_f64(cudaStream_t st, int64_t n, const SegList& S, const double* C, int64_t ldc,
               int m, double alpha, double beta, const SegList& Y0, const OutList& Y);
// colexp (device, s ints, may be nullptr): column k of S is scaled by 2^-colexp[k]
// and row k of C by 2^colexp[k] (exact), so that column scalings of S that C
// undoes (e.g. the D of Rayleigh-Ritz) do not cost fixed-point precision.
// nullptr: the exponents are taken from a column pass over S.
int update_ozaki(cudaStream_t st, int64_t n, const SegList& S, const double* C, int64_t ldc,
                 int m, double alpha, double beta, const SegList& Y0, const OutList& Y,
                 int slices, void* work, int64_t work_bytes, const int* colexp = nullptr);
int64_t update_ozaki_workspace(int64_t n, int s, int m, int slices);

// Residual / preconditioner / Eq. (9) norms for columns c0..m-1; the
// preconditioner enters as its reciprocal diagonal kinv (nullptr: K = I).
// partial: device scratch of residual_workspace(n, m) bytes.
int64_t residual_workspace(int64_t n, int m);
// xb != 0: the column norm in the denominator is sqrt(x^T B x) instead of
// ||x|| (criterion (8) of Sec. 4.3, with normA = 0 and normB = 1).
int residual(cudaStream_t st, int64_t n, const double* X, const double* AX, const double* BX,
             int64_t ld, int m, int c0, const double* theta, const double* kinv, double* W,
             int64_t ldw, double normA, double normB, double* be, void* partial, int xb = 0);
// out = 1 / d (n values)
int reciprocal(cudaStream_t st, int64_t n, const double* d, double* out);

// Column sums of squares of an n x m block: out[j] = sum_i Y(i, j)^2 (fixed order).
int64_t colsumsq_workspace(int64_t n, int m);
int colsumsq(cudaStream_t st, int64_t n, const double* Y, int64_t ld, int m, double* out,
             void* partial);

// out[k] = floor(log2(G_kk)/2) for a Gram G (column-major, leading dim ldg).
int diag_exponents(cudaStream_t st, int n, const double* G, int64_t ldg, int* out);

// Y = diag(b) X (n x m).
int diag_scale(cudaStream_t st, int64_t n, int m, const double* b, const double* X,
               int64_t ldx, double* Y, int64_t ldy);

// Philox4x32-10 normals (see lobpcg_philox_normal).
int philox_normal(cudaStream_t st, int64_t n, int m, uint64_t seed, uint32_t stream_id,
                  double* Y, int64_t ldy);

// Copy an n x m row-major block between leading dimensions (device to device).
int copy_block(cudaStream_t st, int64_t n, int m, const double* X, int64_t ldx, double* Y,
               int64_t ldy);

// Sign normalisation: flip column j so its largest-|.| entry (lowest row on ties)
// is positive.  work: 2 * m * 152 doubles + m ints of scratch.
int sign_normalise(cudaStream_t st, int64_t n, int m, double* X, int64_t ldx, void* work);
int64_t sign_normalise_workspace(int64_t n, int m);

}  // namespace lob

namespace lob {

// ---- eigenpair adjoint (adjoint.cu); column reductions use `partial` of
// adj_reduce_workspace(k) bytes and are fixed-order (deterministic).
int64_t adj_reduce_workspace(int k);
// Cin(j, i) = M(j, i) / (lam_i - lam_j) for j != i; *flag = 1 if a gap < gap.
int adj_coeff(cudaStream_t st, int k, const double* M, int64_t ldm, const double* lam, double gap,
              double* Cin, int* flag);
// Q -= (B P) diag(lam) (BP given, or diagonal b, or B = I); out_j = P_j^T Q_j.
int shift_dot(cudaStream_t st, int64_t n, int k, double* Q, const double* P, const double* BP,
              const double* b, int64_t ld, const double* lam, double* out, void* partial);
// alpha = rz/pq: V -= alpha P, R -= alpha Q, Z = R kinv (kinv null: Z = R), rr = |R_j|^2.
int cg_step(cudaStream_t st, int64_t n, int k, double* V, const double* P, double* R,
            const double* Q, double* Z, const double* kinv, int64_t ld, const double* rz,
            const double* pq, double* rr, void* partial);
int coldot(cudaStream_t st, int64_t n, int k, const double* X, const double* Y, int64_t ld,
           double* out, void* partial);
// P = Z + (rz_new / rz_old) P
int cg_direction(cudaStream_t st, int64_t n, int k, double* P, const double* Z, int64_t ld,
                 const double* rz_new, const double* rz_old);
// coefficient vectors of the A and B gradients (see adjoint.cu)
int grad_coeff(cudaStream_t st, int k, const double* lam, const double* glam, const double* M,
               int64_t ldm, double* caA, double* cwA, double* caB, double* cwB);
int pattern_grad(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* col,
                 const double* X, const double* W, int64_t ld, int k, const double* ca,
                 const double* cw, double* out);
int diag_grad(cudaStream_t st, int64_t n, const double* X, const double* W, int64_t ld, int k,
              const double* ca, const double* cw, double* out);

}  // namespace lob
