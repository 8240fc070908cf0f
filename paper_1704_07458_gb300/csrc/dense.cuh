// Small dense layer (O(n_s^3) work on n_s x n_s matrices, column-major, FP64):
// Rayleigh-Ritz (Algorithms 2 and 7), the svqb / svqbDrop transforms
// (Algorithms 4 and 6) and the Frobenius tests of Algorithm 5.  Factorisations
// run through cuSOLVER/cuBLAS on the device; the decisions that shape the next
// step (Cholesky success, cond(R), how many columns survive) come back to the
// host as a few scalars.
#pragma once
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <vector>

#include "common.cuh"

namespace lob {

// Device-resident path (dense_dev.cu): projected pencils of order <= 256.
constexpr int kDevDenseMax = 256;

struct DevDense {
  int nmax = 0;
  std::vector<void*> bufs;
  double *X = nullptr, *X1 = nullptr, *E = nullptr, *Zt = nullptr;  // nmax x nmax
  double *T1 = nullptr, *T2 = nullptr, *T3 = nullptr, *T4 = nullptr;
  double *XA = nullptr, *GS = nullptr;  // nmax x 2 nmax: [X | A X], [G | S]
  float *V32 = nullptr, *Y32 = nullptr;  // nmax x nmax FP32
  float* f32v = nullptr;                 // 4 nmax FP32 vectors
  double* vec = nullptr;                 // 8 nmax
  double* scal = nullptr;                // 16 device scalars
  int* ints = nullptr;                   // flags, permutation, cluster runs
  double* part = nullptr;                // GEMM split-K partial tiles
  unsigned* cnt = nullptr;               // GEMM split-K tile counters (zero between launches)
  int cnt_tiles = 0;
  int init(int64_t n_max);
  void release();
};

struct DenseLayer {
  cudaStream_t st = nullptr;
  cusolverDnHandle_t sol = nullptr;
  cublasHandle_t blas = nullptr;
  int64_t nmax = 0;
  double* work = nullptr;
  int lwork = 0;
  int* info = nullptr;
  double* A[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // nmax x nmax each
  double* ev = nullptr;    // nmax
  double* d = nullptr;     // nmax
  double* tau = nullptr;   // nmax
  double* scal = nullptr;  // 16 device scalars
  double* host = nullptr;  // pinned host mirror, nmax + 64 doubles
  int64_t launches = 0;
  int64_t syncs = 0;  // host waits on the stream
  // projected eigenproblems: 0 = the device-resident layer of dense_dev.cu
  // for orders <= kDevDenseMax (cuSOLVER FP64 syevd above, and as the
  // fallback when its residual check fails), 1 = FP32 cuSOLVER syevd refined
  // to FP64 (Ogita-Aishima steps, Newton-Schulz, cluster Jacobi, residual
  // check with FP64 fallback), 2 = cuSOLVER FP64 syevd throughout
  int eig_mode = 0;
  int64_t dev_calls = 0, dev_fallbacks = 0;  // device-path eigensolves and their fallbacks
  int64_t check_fail[3] = {0, 0, 0};         // failed checks: orthogonality, wide run, non-finite
  DevDense dev;
  int64_t eig_calls = 0, eig_fallbacks = 0;
  double* R[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // refinement blocks
  float *Af = nullptr, *wf = nullptr, *swork = nullptr;
  int lswork = 0;
  double* part = nullptr;  // norm partials of the refinement
  int* dint = nullptr;     // device permutation, cluster runs, run ids (4 nmax)
  int* hint = nullptr;     // pinned host mirror of dint

  int init(cudaStream_t stream, int64_t n_max);
  void release();
};

// Algorithm 2 on the Gram pair (GA, GB), nx x nx column-major (leading dim nx).
// Writes C (nx x nx, leading dim nx) and theta (device, nx).  *breakdown is set
// when the Cholesky factorisation fails or D GB D is numerically singular.
int rr_initial(DenseLayer& L, const double* GA, const double* GB, int nx, double* C,
               double* theta, bool* breakdown);

// Algorithm 7.  SAS, SBS: ns x ns column-major (leading dim ns).  On success
// writes C = [C_x, C_p] (ns x (nx + *npn), leading dim ns), theta (device, nx)
// and PAP (npn x npn, leading dim npn).  *flip reports the switch to the
// orthogonal branch (Cholesky failure or cond(R)^-3 < tau_skip).
// np: columns of P in S = [X, P, W].  structured: S^T B S came from the
// identities (12)-(13) and is the identity outside the W columns, which the
// device path uses (only the W-block Schur complement is factored); false
// when every block was computed explicitly.
int rr_modified(DenseLayer& L, const double* SAS, const double* SBS, int ns, int nx, int np,
                int nc, bool use_ortho, double tau_skip, bool* flip, double* condR, double* C,
                int* npn, double* theta, double* PAP, bool structured = true);

// Rayleigh-Ritz of the Hetmaniuk-Lehoucq basis selection (the comparison
// variants of Sec. 6): S is B-orthonormal, eig(S^T A S) = Z Theta Z^T,
// C_x = Z(:, 0:nx), C_p = the svqb orthonormalisation (Algorithm 4) of
// [0; Z_2(:, nc:nx)] - Z_x Z_x^T [0; Z_2(:, nc:nx)] (Eq. 6), P^T A P =
// C_p^T S^T A S C_p.  Same outputs as rr_modified.
int rr_hl(DenseLayer& L, const double* SAS, int ns, int nx, int nc, double* C, int* npn,
          double* theta, double* PAP);

// svqb (drop == false, Algorithm 4) or svqbDrop (drop == true, Algorithm 6) on
// the Gram G = U^T B U (nu x nu, leading dim nu): T = D Z(:, J) Theta(J)^-1/2,
// written nu x *nkeep with leading dim nu.
int svqb_transform(DenseLayer& L, const double* G, int nu, bool drop, double tau, double* T,
                   int* nkeep);

// Assemble the projected pencil on S = [X, P, W] from Theta, the saved P^T A P
// (Eq. 14), the identities (12)-(13) and the W columns GAw = S^T A W,
// GBw = S^T B W (ns x nw, leading dim ldgw; GBw == nullptr: S^T B S = I).
// c0 (default nx + np, the W columns): first column of S^T A S, S^T B S that
// GAw, GBw hold (ns x (ns - c0)); the blocks left of and above c0 come from
// the identities.
int assemble(DenseLayer& L, int nx, int np, int nw, const double* theta, const double* PAP,
             int ldpap, const double* GAw, const double* GBw, int ldgw, double* SAS,
             double* SBS, int c0 = -1);

// out[0] = ||G - I||_F (identity == true) or ||G||_F; out[1] = sum(a[0:na]);
// out[2] = sum(b[0:nb]).  G: rows x cols, leading dim ldg.  Result to host.
int small_stats(DenseLayer& L, const double* G, int rows, int cols, int ldg, bool identity,
                const double* a, int na, const double* b, int nb, double out[3]);

// ---- device-resident path (dense_dev.cu)
// C = alpha op(A) op(B) + beta Cin, column-major, m, n <= 2 * the layer's
// order; skip: device flag, the launch is a no-op when it is non-zero.
int dev_gemm(DenseLayer& L, bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
             int lda, const double* B, int ldb, double beta, const double* Cin, int ldcin,
             double* C, int ldc, const int* skip);
int dev_chol(DenseLayer& L, int n, double* A, int lda, int* info);
int dev_trinv(DenseLayer& L, int n, const double* R, int ldr, double* X, int ldx, const int* skip);
int dev_syev(DenseLayer& L, int n, const double* A, int lda, double* Z, int ldz, double* w,
             int* status);
int dev_syev_refine(DenseLayer& L, int n, double* Z, int ldz, double* w, int* status, int steps);
int dev_orth_basis(DenseLayer& L, int m, int c, const double* M, int ldm, double* Q, int ldq);
bool dev_rr_fits(const DenseLayer& L, int ns, int nx, int nw);
int rr_initial_dev(DenseLayer& L, const double* GA, const double* GB, int nx, double* C,
                   double* theta, bool* breakdown);
int rr_modified_dev(DenseLayer& L, const double* SAS, const double* SBS, int ns, int nx, int np,
                    int nc, bool use_ortho, double tau_skip, bool* flip, double* condR, double* C,
                    int* npn, double* theta, double* PAP);
bool dev_explicit_fits(const DenseLayer& L, int ns, int nx, int np);
int rr_explicit_dev(DenseLayer& L, const double* SAS, const double* SBS, int ns, int nx, int np,
                    int nc, double tau_skip, bool* flip, double* condR, double* C, int* npn,
                    double* theta, double* PAP);
int svqb_transform_dev(DenseLayer& L, const double* G, int nu, bool drop, double tau, double* T,
                       int* nkeep);
// cuSOLVER FP64 eigendecomposition in place (A: eigenvectors, L.ev: eigenvalues)
int syevd_fallback(DenseLayer& L, int n, double* A, int lda);

}  // namespace lob
