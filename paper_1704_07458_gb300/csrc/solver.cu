// Host driver of the robust LOBPCG (Algorithm 8 of Duersch, Shao, Yang, Gu,
// 2018) and the solver half of the C ABI.
//
// Every n-scaled step runs in this library's kernels (spmm.cu, blas.cu,
// ozaki.cu); the O(n_s^3) Rayleigh-Ritz work runs in dense.cu.  The host only
// keeps the control flow: the shapes of the next step depend on a few scalars
// (Cholesky success, cond(R), surviving columns, the number of converged
// pairs) that come back once or a few times per iteration.
//
// Device layout: every n x . block (X, P, W, AX, AP, AW, BX, BP, BW and their
// next-iteration copies) is a separate row-major n x ld buffer, ld = n_x
// rounded up to 8 doubles (64 bytes).  S = [X, P, W] is never materialised:
// the kernels take it as a list of column segments.  The update of Eq. (10)
// writes into the "next" buffers and the pointers swap (ping-pong), which
// the paper's row-chunked in-place scheme of Eq. (11) needs no workspace for.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dense.cuh"
#include "kernels.cuh"

using namespace lob;

namespace {
constexpr double kEps = 2.220446049250313e-16;

enum Phase { PH_SPMM, PH_GRAM, PH_UPDATE, PH_RESID, PH_DENSE, PH_ORTHO, PH_OTHER, PH_COUNT };

struct PhaseTimer {
  // Exclusive accounting on the stream: every phase boundary records an event
  // and the interval since the previous boundary is charged to the innermost
  // open phase, or to PH_OTHER when no phase is open.  The totals therefore
  // add up to the stream time between the first and the last boundary.
  std::vector<cudaEvent_t> pool;
  struct Seg { int phase; int e0, e1; };
  std::vector<Seg> segs;
  std::vector<int> open;  // phase stack
  int last = -1;          // event of the previous boundary
  size_t used = 0;
  double total[PH_COUNT] = {0};
  cudaStream_t st = nullptr;
  int ev() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    cudaEventRecord(pool[used], st);
    return (int)used++;
  }
  void mark() {
    const int e = ev();
    if (last >= 0) segs.push_back({open.empty() ? PH_OTHER : open.back(), last, e});
    last = e;
  }
  void begin(int ph) {
    mark();
    open.push_back(ph);
  }
  void end() {
    mark();
    open.pop_back();
  }
  // Call only after a stream synchronisation.
  void flush() {
    for (auto& m : segs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pool[m.e0], pool[m.e1]) == cudaSuccess) total[m.phase] += ms;
    }
    segs.clear();
    if (last >= 0) {  // keep only the last boundary's event
      std::swap(pool[0], pool[last]);
      last = 0;
      used = 1;
    } else {
      used = 0;
    }
  }
  void reset() {
    segs.clear();
    open.clear();
    last = -1;
    used = 0;
    for (auto& t : total) t = 0;
  }
  ~PhaseTimer() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct Scoped {
  PhaseTimer& t;
  Scoped(PhaseTimer& tm, int ph) : t(tm) { t.begin(ph); }
  ~Scoped() { t.end(); }
};
}  // namespace

struct lobpcg_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  lobpcg_options_t opt{};
  std::string err;
  lobpcg_stats_t stats{};
  // operator
  int64_t n = 0, A_nnz = 0, B_nnz = 0;
  int32_t *A_rp = nullptr, *A_ci = nullptr, *B_rp = nullptr, *B_ci = nullptr;
  // operator arrays used in place (lobpcg_set_operator_ex with LOBPCG_BORROW):
  // bit 0 A_rp, 1 A_ci, 2 A_v, 3 B_rp, 4 B_ci, 5 B_v; never freed here
  unsigned borrowed = 0;
  double *A_v = nullptr, *B_v = nullptr, *b_diag = nullptr;
  int b_kind = 0;  // 0 identity, 1 diagonal, 2 CSR
  double b_cond = 1.0;
  int k_kind = 0;  // 0 diag(A), 1 user diagonal, 2 identity, 3 callback
  double *adiag = nullptr, *kdiag = nullptr;
  lobpcg_precond_fn cb = nullptr;
  void* cb_ctx = nullptr;
  // workspace of the current shape
  std::vector<void*> ws;
  int64_t ws_n = -1, ws_nx = -1;
  int ws_b = -1, ws_mode = -1, ws_slices = -1;
  int64_t ld = 0;
  double *X, *P, *AX, *AP, *AW, *BX, *BP, *BW, *Xn, *Pn, *AXn, *APn, *BXn, *BPn, *Om;
  double* wbuf[4];
  double *theta, *be, *colA, *colB, *Gw, *Gs, *SAS, *SBS, *Cm, *PAP, *PAPn;
  double* kinv = nullptr;  // 1 / diag(K) for the current solve (n)
  int slice_boost = 0;     // 7 once a solve in an emulated form has stalled
  int *cexp, *zexp;  // column balance exponents of S, and all zeros
  int* dstatus = nullptr;  // device status word of the tensor-core kernels (bit 0: a wait ran out)
  void* gwork = nullptr;
  int64_t gwork_bytes = 0;
  void* uwork = nullptr;
  int64_t uwork_bytes = 0;
  void* rwork = nullptr;
  double* hbuf = nullptr;  // pinned host
  int64_t syncs = 0;       // host waits on the stream (stats.host_syncs)
  DenseLayer dense;
  PhaseTimer timer;

  ~lobpcg_ctx() { release_all(); }

  void free_ws() {
    for (void* p : ws) cudaFree(p);
    ws.clear();
    ws_n = ws_nx = -1;
  }
  void release_op() {
    int bit = 0;
    for (void** p : {(void**)&A_rp, (void**)&A_ci, (void**)&A_v, (void**)&B_rp, (void**)&B_ci,
                     (void**)&B_v, (void**)&b_diag, (void**)&adiag, (void**)&kdiag}) {
      if (*p && !((borrowed >> bit) & 1u)) cudaFree(*p);
      *p = nullptr;
      ++bit;
    }
    borrowed = 0;
  }
  void release_all() {
    free_ws();
    release_op();
    dense.release();
    if (hbuf) cudaFreeHost(hbuf);
    hbuf = nullptr;
  }
  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
};

namespace {

int dalloc(lobpcg_ctx* h, void** p, size_t bytes) {
  if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    return LOBPCG_ERR_OOM;
  }
  h->ws.push_back(*p);
  return LOBPCG_OK;
}

int gemm_mode(const lobpcg_ctx* h) {
  return (h->opt.gemm_mode == LOBPCG_GEMM_OZAKI || h->opt.gemm_mode == LOBPCG_GEMM_OZAKI_TC)
             ? h->opt.gemm_mode
             : 0;
}
// Slices of the emulated contractions: the option (default 6), raised to 7
// for the rest of a solve when the iteration stalls (see solve_impl).
int slices(const lobpcg_ctx* h) {
  const int sl = h->opt.ozaki_slices > 0 ? h->opt.ozaki_slices : 6;
  return std::max(sl, h->slice_boost);
}

int ensure_workspace(lobpcg_ctx* h, int64_t nx) {
  const int64_t n = h->n;
  if (h->ws_n == n && h->ws_nx == nx && h->ws_b == h->b_kind && h->ws_mode == gemm_mode(h) &&
      h->ws_slices == slices(h))
    return LOBPCG_OK;
  h->free_ws();
  const int s = h->opt.omega_rows > 0 ? h->opt.omega_rows : 16;
  h->ld = round_up(std::max<int64_t>(nx, s), 8);
  const size_t blk = (size_t)n * h->ld * sizeof(double);
  int rc;
  double** blocks[] = {&h->X, &h->P, &h->AX, &h->AP, &h->AW, &h->Xn, &h->Pn, &h->AXn, &h->APn,
                       &h->wbuf[0], &h->wbuf[1], &h->wbuf[2], &h->wbuf[3], &h->Om};
  for (double** b : blocks)
    if ((rc = dalloc(h, (void**)b, blk))) return rc;
  if (h->b_kind != 0) {
    double** bb[] = {&h->BX, &h->BP, &h->BW, &h->BXn, &h->BPn};
    for (double** b : bb)
      if ((rc = dalloc(h, (void**)b, blk))) return rc;
  } else {
    h->BX = h->BP = h->BW = h->BXn = h->BPn = nullptr;
  }
  const int64_t nsmax = 3 * nx;
  const size_t sm = (size_t)nsmax * nsmax * sizeof(double);
  double** smalls[] = {&h->Gw, &h->Gs, &h->SAS, &h->SBS, &h->Cm, &h->PAP, &h->PAPn};
  for (double** b : smalls)
    if ((rc = dalloc(h, (void**)b, 2 * sm))) return rc;
  double** vecs[] = {&h->theta, &h->be, &h->colA, &h->colB};
  for (double** b : vecs)
    if ((rc = dalloc(h, (void**)b, (size_t)std::max<int64_t>(nsmax, s) * 2 * sizeof(double))))
      return rc;
  if ((rc = dalloc(h, (void**)&h->kinv, (size_t)n * sizeof(double)))) return rc;
  if ((rc = dalloc(h, (void**)&h->cexp, (size_t)nsmax * sizeof(int)))) return rc;
  if ((rc = dalloc(h, (void**)&h->zexp, (size_t)nsmax * sizeof(int)))) return rc;
  if ((rc = dalloc(h, (void**)&h->dstatus, 16))) return rc;
  LOB_CUDA_OK(cudaMemsetAsync(h->zexp, 0, (size_t)nsmax * sizeof(int), h->st));
  // Gram scratch: the widest uses are S^T [AW, BW] (3 nx x 2 nx) and, when
  // every block is computed (CHL, the explicit Rayleigh-Ritz), S^T A S and
  // S^T B S (3 nx x 3 nx each).
  const int mode = gemm_mode(h), sl = slices(h);
  // The slab count depends on the shape, so take the maximum over every Gram
  // shape the driver can request (p <= 3 n_x, q <= 3 n_x).
  int64_t gb = 0;
  for (int p = 1; p <= nsmax; ++p)
    for (int q = 1; q <= nsmax; ++q) {
      gb = std::max(gb, gram_f64_workspace(n, p, q));
      if (mode) gb = std::max(gb, gram_ozaki_workspace(n, p, q, std::max(sl, 7)));
      if (mode == LOBPCG_GEMM_OZAKI_TC) gb = std::max(gb, gram_tc_workspace(n, p, q));
    }
  h->gwork_bytes = gb;
  if ((rc = dalloc(h, &h->gwork, (size_t)gb))) return rc;
  h->uwork_bytes = mode ? update_ozaki_workspace(n, (int)nsmax, (int)(2 * nx), std::max(sl, 7)) : 0;
  if (mode == LOBPCG_GEMM_OZAKI_TC)  // the tile split depends on m: take every m
    for (int m = 1; m <= 2 * nx; ++m)
      h->uwork_bytes = std::max({h->uwork_bytes, update_tc_workspace(n, (int)nsmax, m, sl),
                                 update_tc_workspace(n, (int)nsmax, m, 7)});
  if (h->uwork_bytes > 0 && (rc = dalloc(h, &h->uwork, (size_t)h->uwork_bytes))) return rc;
  const int64_t rb = std::max(residual_workspace(n, (int)h->ld), colsumsq_workspace(n, (int)h->ld));
  if ((rc = dalloc(h, &h->rwork, (size_t)rb))) return rc;
  if ((rc = h->dense.init(h->st, nsmax))) return rc;
  h->dense.eig_mode = (h->opt.dense_eig == 1 || h->opt.dense_eig == 2) ? h->opt.dense_eig : 0;
  h->ws_n = n;
  h->ws_nx = nx;
  h->ws_b = h->b_kind;
  h->ws_mode = mode;
  h->ws_slices = sl;
  return LOBPCG_OK;
}

// ---- thin wrappers choosing the arithmetic of the dense contractions

// min_slices: the orthogonality tests of Algorithm 5 compare ||U^T B U - I||
// with 100 eps, which needs the 7-slice (2^-56) split; the projected pencil
// does not.
int gram(lobpcg_ctx* h, const SegList& U, const SegList& V, double* G, int64_t ldg,
         int min_slices = 0) {
  Scoped sc(h->timer, PH_GRAM);
  h->stats.gram_calls++;
  h->stats.gram_flops += 2.0 * h->n * U.off[U.nseg] * V.off[V.nseg];
  h->stats.gram_bytes += 8.0 * h->n * (U.off[U.nseg] + V.off[V.nseg]);
  if (gemm_mode(h)) {
    const int sl = std::max(slices(h), min_slices);
    h->stats.gram_tensor_flops += 2.0 * h->n * U.off[U.nseg] * V.off[V.nseg] * sl * (sl + 1) / 2;
  }
  if (gemm_mode(h) == LOBPCG_GEMM_OZAKI_TC)
    return gram_tc(h->st, h->n, U, V, G, ldg, std::max(slices(h), min_slices), h->gwork,
                   h->gwork_bytes);
  if (gemm_mode(h))
    return gram_ozaki(h->st, h->n, U, V, G, ldg, std::max(slices(h), min_slices), h->gwork,
                      h->gwork_bytes);
  return gram_f64(h->st, h->n, U, V, G, ldg, h->gwork, h->gwork_bytes);
}

// colexp: per-column power-of-two balance of S for the tensor-core path (see
// update_ozaki); h->zexp when the columns of S are already balanced.
int update(lobpcg_ctx* h, const SegList& S, const double* C, int64_t ldc, int m, double alpha,
           double beta, const SegList& Y0, const OutList& Y, const int* colexp,
           int min_slices = 0) {
  Scoped sc(h->timer, PH_UPDATE);
  h->stats.update_calls++;
  h->stats.update_flops += 2.0 * h->n * S.off[S.nseg] * m;
  h->stats.update_bytes += 8.0 * h->n * (S.off[S.nseg] + m + (beta != 0.0 ? m : 0));
  if (gemm_mode(h)) {
    const int sl = std::max(slices(h), min_slices);
    h->stats.update_tensor_flops += 2.0 * h->n * S.off[S.nseg] * m * sl * (sl + 1) / 2;
  }
  if (gemm_mode(h) == LOBPCG_GEMM_OZAKI_TC)
    return update_tc(h->st, h->n, S, C, ldc, m, alpha, beta, Y0, Y,
                     std::max(slices(h), min_slices), h->uwork, h->uwork_bytes, colexp,
                     h->dstatus);
  if (gemm_mode(h))
    return update_ozaki(h->st, h->n, S, C, ldc, m, alpha, beta, Y0, Y,
                        std::max(slices(h), min_slices), h->uwork, h->uwork_bytes, colexp);
  return update_f64(h->st, h->n, S, C, ldc, m, alpha, beta, Y0, Y);
}

OutList out1(double* p, int64_t ld, int m) { return OutList{{p, p}, {ld, ld}, m}; }

// Y = A X (and BY = B X when by != nullptr and B is not the identity)
int apply_AB(lobpcg_ctx* h, const double* X, int m, double* AY, double* BY) {
  if (m <= 0) return LOBPCG_OK;
  Scoped sc(h->timer, PH_SPMM);
  const double n = (double)h->n;
  h->stats.spmm_calls++;
  h->stats.spmm_bytes += h->A_nnz * 12.0 + 4.0 * (n + 1) + 16.0 * n * m +
                         ((BY && h->b_kind == 1) ? 8.0 * n + 16.0 * n * m : 0.0);
  // the diagonal-B product rides along with A X; a sparse B gets its own pass
  const bool fused = BY && h->b_kind == 1;
  int rc = spmm(h->st, h->n, h->A_rp, h->A_ci, h->A_v, X, h->ld, m, AY, h->ld,
                fused ? h->b_diag : nullptr, fused ? BY : nullptr, h->ld);
  if (rc || !BY) return rc;
  if (h->b_kind == 2)
    rc = spmm(h->st, h->n, h->B_rp, h->B_ci, h->B_v, X, h->ld, m, BY, h->ld, nullptr, nullptr, 0);
  return rc;
}

int apply_B(lobpcg_ctx* h, const double* X, int m, double* BY) {
  if (m <= 0 || h->b_kind == 0) return LOBPCG_OK;
  Scoped sc(h->timer, PH_SPMM);
  if (h->b_kind == 1) return diag_scale(h->st, h->n, m, h->b_diag, X, h->ld, BY, h->ld);
  return spmm(h->st, h->n, h->B_rp, h->B_ci, h->B_v, X, h->ld, m, BY, h->ld, nullptr, nullptr, 0);
}

int to_host(lobpcg_ctx* h, double* dst, const double* src, int64_t count) {
  if (count <= 0) return LOBPCG_OK;
  LOB_CUDA_OK(cudaMemcpyAsync(h->hbuf, src, count * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  LOB_CUDA_OK(cudaStreamSynchronize(h->st));
  ++h->syncs;
  memcpy(dst, h->hbuf, count * sizeof(double));
  h->timer.flush();
  return LOBPCG_OK;
}

// Backward errors of the current iterate and the tensor-core status word in
// one host wait; a bounded wait that ran out in a tensor-core kernel turns
// into LOBPCG_ERR_TIMEOUT (its outputs are not valid).
int read_be(lobpcg_ctx* h, double* dst, int64_t count) {
  if (count > 0)
    LOB_CUDA_OK(cudaMemcpyAsync(h->hbuf, h->be, count * sizeof(double), cudaMemcpyDeviceToHost,
                                h->st));
  LOB_CUDA_OK(cudaMemcpyAsync(h->hbuf + std::max<int64_t>(count, 0) + 1, h->dstatus, sizeof(int),
                              cudaMemcpyDeviceToHost, h->st));
  LOB_CUDA_OK(cudaStreamSynchronize(h->st));
  ++h->syncs;
  if (count > 0) memcpy(dst, h->hbuf, count * sizeof(double));
  int stw = 0;
  memcpy(&stw, h->hbuf + std::max<int64_t>(count, 0) + 1, sizeof(int));
  h->timer.flush();
  return stw ? h->fail(LOBPCG_ERR_TIMEOUT, "a tensor-core kernel's bounded wait ran out") : 0;
}

int sum_sq_norms(lobpcg_ctx* h, const double* Y, int m, double* out) {
  // out = sum of squares of an n x m block
  int rc = colsumsq(h->st, h->n, Y, h->ld, m, h->colA, h->rwork);
  if (rc) return rc;
  double s[3];
  if ((rc = small_stats(h->dense, h->Gs, 0, 0, 1, false, h->colA, m, h->colA, 0, s))) return rc;
  *out = s[1];
  return LOBPCG_OK;
}

int64_t leading_converged(const double* be, int64_t m, double tol) {
  int64_t i = 0;
  while (i < m && be[i] <= tol) ++i;
  return i;
}

// Algorithm 5 (orthoDrop) with M = B on the active W columns.  U points at the
// active block (inside one of the wbuf buffers); the result may move to another
// buffer.  V = [X, P] with BV = [BX, BP].
// drop == false: Algorithm 3 (svqb on every inner pass, no column dropped),
// the orthogonalisation of the Hetmaniuk-Lehoucq comparison variants.
int ortho_drop(lobpcg_ctx* h, double*& U, double*& Ubase, int& nu, int nx, int np,
               double tau_ortho, bool drop = true) {
  Scoped sc(h->timer, PH_ORTHO);
  h->stats.ortho_calls++;
  const int nin = nu;
  auto spare = [&](const double* a, const double* b) {
    for (double* w : h->wbuf)
      if (w != a && w != b) return w;
    return (double*)nullptr;
  };
  const double* BXp = h->b_kind ? h->BX : h->X;
  const double* BPp = h->b_kind ? h->BP : h->P;
  SegList V = seg_empty();
  seg_push(V, h->X, h->ld, nx);
  seg_push(V, h->P, h->ld, np);
  SegList BV = seg_empty();
  seg_push(BV, BXp, h->ld, nx);
  seg_push(BV, BPp, h->ld, np);
  const int nv = nx + np;
  int rc;
  double nbv = 0.0, t;
  if ((rc = sum_sq_norms(h, BXp, nx, &nbv))) return rc;
  if (np > 0) {
    if ((rc = sum_sq_norms(h, BPp, np, &t))) return rc;
    nbv += t;
  }
  nbv = std::sqrt(nbv);
  double* BU = h->b_kind ? h->BW : nullptr;
  double st3[3];
  for (int i = 0; i < 3 && nu > 0; ++i) {
    // U = U - V (V^T B U), with V^T B U formed as (BV)^T U
    if ((rc = gram(h, BV, seg1(U, h->ld, nu), h->Gs, nv, 7))) return rc;
    double* dst = spare(Ubase, nullptr);
    if ((rc = update(h, V, h->Gs, nv, nu, -1.0, 1.0, seg1(U, h->ld, nu), out1(dst, h->ld, nu),
                     h->zexp, 7)))
      return rc;
    U = Ubase = dst;
    for (int j = 0; j < 3; ++j) {
      const double* BUp = U;
      if (h->b_kind) {
        if ((rc = apply_B(h, U, nu, BU))) return rc;
        BUp = BU;
      }
      if ((rc = gram(h, seg1(U, h->ld, nu), seg1(BUp, h->ld, nu), h->Gs, nu, 7))) return rc;
      if ((rc = diag_exponents(h->st, nu, h->Gs, nu, h->cexp))) return rc;
      int keep = 0;
      {
        Scoped sd(h->timer, PH_DENSE);
        if ((rc = svqb_transform(h->dense, h->Gs, nu, drop && j > 0, nu * kEps, h->Cm, &keep)))
          return rc;
      }
      h->stats.svqb_passes++;
      if (keep == 0) {
        nu = 0;
        break;
      }
      dst = spare(Ubase, nullptr);
      if ((rc = update(h, seg1(U, h->ld, nu), h->Cm, nu, keep, 1.0, 0.0, seg_empty(),
                       out1(dst, h->ld, keep), h->cexp, 7)))
        return rc;
      U = Ubase = dst;
      nu = keep;
      BUp = U;
      if (h->b_kind) {
        if ((rc = apply_B(h, U, nu, BU))) return rc;
        BUp = BU;
      }
      if ((rc = gram(h, seg1(U, h->ld, nu), seg1(BUp, h->ld, nu), h->Gs, nu, 7))) return rc;
      if ((rc = colsumsq(h->st, h->n, U, h->ld, nu, h->colA, h->rwork))) return rc;
      if ((rc = colsumsq(h->st, h->n, BUp, h->ld, nu, h->colB, h->rwork))) return rc;
      if ((rc = small_stats(h->dense, h->Gs, nu, nu, nu, true, h->colA, nu, h->colB, nu, st3)))
        return rc;
      const double err = st3[0] / (std::sqrt(st3[2]) * std::sqrt(st3[1]));
      if (err <= tau_ortho) break;
    }
    if (nu == 0 || nv == 0) break;
    if ((rc = gram(h, BV, seg1(U, h->ld, nu), h->Gs, nv, 7))) return rc;
    if ((rc = colsumsq(h->st, h->n, U, h->ld, nu, h->colA, h->rwork))) return rc;
    if ((rc = small_stats(h->dense, h->Gs, nv, nu, nv, false, h->colA, nu, h->colA, 0, st3)))
      return rc;
    const double err = st3[0] / (nbv * std::sqrt(st3[1]));
    if (err <= tau_ortho) break;
  }
  h->stats.dropped_columns += nin - nu;
  return LOBPCG_OK;
}

int solve_impl(lobpcg_ctx* h, int64_t k, double tol, const double* X0, int64_t ldx0,
               uint64_t seed, int mem_in, double* lambda, double* Xout, int64_t ldx,
               int mem_out, int64_t* iters, double* resnorm) {
  const int64_t n = h->n;
  if (n <= 0) return h->fail(LOBPCG_ERR_ARG, "no operator set");
  if (k <= 0 || k > n) return h->fail(LOBPCG_ERR_ARG, "k must be in 1..n");
  if (!(tol > 0)) return h->fail(LOBPCG_ERR_ARG, "tol must be positive");
  int64_t nx = h->opt.block_width > 0 ? h->opt.block_width
                                      : k + std::max<int64_t>((k + 9) / 10, 2);
  nx = std::min(nx, n);
  if (nx < k) return h->fail(LOBPCG_ERR_ARG, "block_width < k");
  if (3 * nx > 6144) return h->fail(LOBPCG_ERR_ARG, "block too wide (3 n_x > 6144)");
  if (!lambda || !Xout || ldx < k) return h->fail(LOBPCG_ERR_ARG, "bad output buffers");
  if (X0 && ldx0 < nx) return h->fail(LOBPCG_ERR_ARG, "ldx0 < block width");
  for (int m : {mem_in, mem_out})
    if (m != LOBPCG_MEM_HOST && m != LOBPCG_MEM_DEVICE)
      return h->fail(LOBPCG_ERR_ARG, "memory kinds must be LOBPCG_MEM_HOST or LOBPCG_MEM_DEVICE");
  if (h->k_kind == 3 && !h->cb) return h->fail(LOBPCG_ERR_ARG, "no callback set");
  h->slice_boost = 0;
  int rc = ensure_workspace(h, nx);
  if (rc) return h->fail(rc, "workspace allocation failed");
  LOB_CUDA_OK(cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
  const auto t_start = std::chrono::steady_clock::now();
  const int64_t launches0 = g_launches;
  const int64_t eig0 = h->dense.eig_calls + h->dense.dev_calls,
                eigf0 = h->dense.eig_fallbacks + h->dense.dev_fallbacks;
  const int64_t syncs0 = h->syncs + h->dense.syncs;
  const int64_t cf0[3] = {h->dense.check_fail[0], h->dense.check_fail[1], h->dense.check_fail[2]};
  h->timer.st = h->st;
  h->timer.reset();
  h->timer.mark();
  h->stats = lobpcg_stats_t{};
  h->stats.n_x = nx;
  h->stats.flip_iteration = -1;
  h->stats.slice_escalation_iteration = -1;
  h->stats.orth_error = -1.0;
  const int64_t ld = h->ld;
  const int s = h->opt.omega_rows > 0 ? h->opt.omega_rows : 16;
  const int maxit = h->opt.maxit > 0 ? h->opt.maxit : 6000;
  const double tau_ortho = h->opt.tau_ortho > 0 ? h->opt.tau_ortho : 100 * kEps;
  const double tau_skip = h->opt.tau_skip > 0 ? h->opt.tau_skip : 100 * kEps;
  const int refresh_every = h->opt.refresh_every > 0 ? h->opt.refresh_every : 50;
  bool implicit = h->b_kind == 0 || (h->b_kind == 1 && h->b_cond <= 1e4);
  if (h->opt.implicit == 1) implicit = false;
  if (h->opt.implicit == 2) implicit = true;
  // basis selection: Algorithm 8, or the Hetmaniuk-Lehoucq comparison
  // variants of Sec. 6 (CHL: no implicit products, every block computed;
  // AHL: implicit products, only (12) assumed)
  const int basis = (h->opt.basis == 1 || h->opt.basis == 2) ? h->opt.basis : 0;
  const bool hl = basis != 0;
  if (basis == 1) implicit = false;
  // explicit Rayleigh-Ritz after refreshes: default on in the emulated forms
  const bool erx = h->opt.explicit_rr == 2 || (h->opt.explicit_rr == 0 && gemm_mode(h) != 0);
  // convergence test: Eq. (9), or the relative residuals (7) / (8)
  const int crit = (h->opt.criterion == 7 || h->opt.criterion == 8) ? h->opt.criterion : 9;
  const double* kd = (h->k_kind == 0) ? h->adiag : (h->k_kind == 1 ? h->kdiag : nullptr);
  if (kd) {
    if ((rc = reciprocal(h->st, n, kd, h->kinv))) return rc;
    kd = h->kinv;  // the residual pass applies K^-1 as a product
  }
  std::vector<double> be_h(std::max<int64_t>(nx, s) + 8), th_h(nx);

  // ---- Sec. 4.3: Gaussian-sketch norm estimates ||M||^(Omega) = ||M Omega^T||_F / ||Omega||_F
  if ((rc = philox_normal(h->st, n, s, seed, 5u, h->Om, ld))) return rc;
  double om2, am2, bm2 = 1.0;
  if ((rc = sum_sq_norms(h, h->Om, s, &om2))) return rc;
  double* tmp = h->wbuf[0];
  if ((rc = apply_AB(h, h->Om, s, tmp, nullptr))) return rc;
  if ((rc = sum_sq_norms(h, tmp, s, &am2))) return rc;
  const double normA = std::sqrt(am2 / om2);
  double normB = 1.0;
  if (h->b_kind) {
    if ((rc = apply_B(h, h->Om, s, tmp))) return rc;
    if ((rc = sum_sq_norms(h, tmp, s, &bm2))) return rc;
    normB = std::sqrt(bm2 / om2);
  }
  h->stats.norm_a = normA;
  h->stats.norm_b = normB;

  // ---- Algorithm 8, initial step: X = X0 C with [C, Theta] = RayleighRitz(X0)
  if (X0) {
    LOB_CUDA_OK(cudaMemcpy2DAsync(h->X, ld * sizeof(double), X0, ldx0 * sizeof(double),
                                  nx * sizeof(double), n,
                                  mem_in == LOBPCG_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                              : cudaMemcpyHostToDevice,
                                  h->st));
  } else if ((rc = philox_normal(h->st, n, (int)nx, seed, 1u, h->X, ld))) {
    return rc;
  }
  double* BXp = h->b_kind ? h->BX : h->X;
  if ((rc = apply_AB(h, h->X, (int)nx, h->AX, h->BX))) return rc;
  {
    Scoped sc(h->timer, PH_GRAM);
    SegList V = seg_empty();
    seg_push(V, h->AX, ld, (int)nx);
    seg_push(V, BXp, ld, (int)nx);
    if ((rc = gram(h, seg1(h->X, ld, (int)nx), V, h->Gw, nx))) return rc;
  }
  if ((rc = diag_exponents(h->st, (int)nx, h->Gw + nx * nx, (int)nx, h->cexp))) return rc;
  bool breakdown = false;
  {
    Scoped sc(h->timer, PH_DENSE);
    if ((rc = rr_initial(h->dense, h->Gw, h->Gw + nx * nx, (int)nx, h->Cm, h->theta, &breakdown)))
      return rc;
  }
  if (breakdown) return h->fail(LOBPCG_ERR_BREAKDOWN, "initial block is rank deficient");
  {
    Scoped sc(h->timer, PH_UPDATE);
    if ((rc = update(h, seg1(h->X, ld, (int)nx), h->Cm, nx, (int)nx, 1.0, 0.0, seg_empty(),
                     out1(h->Xn, ld, (int)nx), h->cexp)))
      return rc;
  }
  std::swap(h->X, h->Xn);
  BXp = h->b_kind ? h->BX : h->X;
  if ((rc = apply_AB(h, h->X, (int)nx, h->AX, h->BX))) return rc;

  int64_t nc = 0;
  int np = 0;
  bool use_ortho = hl, refresh_next = false, explicit_next = false;
  constexpr int64_t kStallWindow = 400;
  int64_t stall_nc = -1, stall_it = 0;
  double stall_be = INFINITY;
  int64_t it = 0;
  int status = LOBPCG_OK;
  // W (or R for a callback preconditioner) of columns c0 .. nx-1, then locking.
  double* Wbase = h->wbuf[0];
  double* Wp = Wbase;
  // criterion (9): ||r|| / ((||A|| + |theta| ||B||) ||x||); (7): ||r|| /
  // (|theta| ||x||); (8): ||r|| / (|theta| ||x||_B)
  const double cA = crit == 9 ? normA : 0.0, cB = crit == 9 ? normB : 1.0;
  auto residual_step = [&](int64_t c0, bool write_w) -> int {
    Scoped sc(h->timer, PH_RESID);
    const double* bx = h->b_kind ? h->BX : nullptr;
    double* dst = nullptr;
    if (write_w) dst = (h->k_kind == 3) ? h->wbuf[3] : Wbase;
    int r = residual(h->st, n, h->X, h->AX, bx, ld, (int)nx, (int)c0, h->theta,
                     (h->k_kind == 3) ? nullptr : kd, dst, ld, cA, cB, h->be, h->rwork,
                     crit == 8 ? 1 : 0);
    return r;
  };
  auto finish_w = [&](int64_t c0, int64_t ncn) -> int {
    // active W columns ncn .. nx-1 of a residual written from column c0
    const int64_t off = ncn - c0;
    if (h->k_kind == 3) {
      const int64_t nw = nx - ncn;
      if (nw > 0 && h->cb(h->cb_ctx, n, nw, h->wbuf[3] + off, ld, Wbase, ld, (void*)h->st) != 0)
        return LOBPCG_ERR_CALLBACK;
      Wp = Wbase;
    } else {
      Wp = Wbase + off;
    }
    return LOBPCG_OK;
  };
  Wbase = h->wbuf[0];
  if ((rc = residual_step(0, true))) return rc;
  if ((rc = read_be(h, be_h.data(), nx))) return rc;
  nc = std::min<int64_t>(leading_converged(be_h.data(), nx, tol), nx);
  if ((rc = finish_w(0, nc))) return h->fail(rc, "preconditioner callback failed");

  for (;;) {
    while (nc < k) {
      if (it >= maxit) {
        status = LOBPCG_ERR_NOT_CONVERGED;
        break;
      }
      if (h->opt.max_seconds > 0 &&
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() >
              h->opt.max_seconds) {
        status = LOBPCG_ERR_TIMEOUT;
        break;
      }
      ++it;
      h->stats.iterations = it;  // also what an error return reports
      int nw = (int)(nx - nc);
      // which blocks of the projected pencil are computed rather than taken
      // from the identities (12)-(14): the W columns (Algorithm 8), P and W
      // (AHL), or all (CHL, and the explicit Rayleigh-Ritz after a refresh)
      const bool direct_all =
          basis == 1 || (explicit_next && !hl) || (basis == 0 && h->opt.gram_blocks == 2);
      if (explicit_next && !hl) h->stats.explicit_rr_calls++;
      // W-products, Grams, projected pencil
      auto project = [&](bool ortho, int c0, bool need_b) -> int {
        int r;
        double* BWp = h->b_kind ? h->BW : Wp;
        if ((r = apply_AB(h, Wp, nw, h->AW, h->b_kind ? h->BW : nullptr))) return r;
        const int ns = (int)nx + np + nw;
        SegList S = seg_empty();
        seg_push(S, h->X, ld, (int)nx);
        seg_push(S, h->P, ld, np);
        seg_push(S, Wp, ld, nw);
        const double* BXp = h->b_kind ? h->BX : h->X;
        const double* BPp = h->b_kind ? h->BP : h->P;
        SegList VA = seg_empty(), VB = seg_empty();
        if (c0 <= 0) {
          seg_push(VA, h->AX, ld, (int)nx);
          seg_push(VB, BXp, ld, (int)nx);
        }
        if (c0 <= (int)nx) {
          seg_push(VA, h->AP, ld, np);
          seg_push(VB, BPp, ld, np);
        }
        seg_push(VA, h->AW, ld, nw);
        seg_push(VB, BWp, ld, nw);
        const int nd = ns - c0;  // computed columns
        const bool with_b = need_b && !ortho;
        {
          Scoped sc(h->timer, PH_GRAM);
          if (c0 == (int)nx + np) {  // one Gram for S^T [A W, B W]
            SegList V = VA;
            if (with_b) seg_push(V, BWp, ld, nw);
            if ((r = gram(h, S, V, h->Gw, ns))) return r;
          } else {
            if ((r = gram(h, S, VA, h->Gw, ns))) return r;
            if (with_b && (r = gram(h, S, VB, h->Gw + (int64_t)ns * nd, ns))) return r;
          }
        }
        Scoped sd(h->timer, PH_DENSE);
        return assemble(h->dense, (int)nx, np, nw, h->theta, h->PAP, np, h->Gw,
                        with_b ? h->Gw + (int64_t)ns * nd : nullptr, ns, h->SAS, h->SBS, c0);
      };
      const bool p_direct = basis == 2 || (basis == 0 && h->opt.gram_blocks == 1);
      const int c0 = direct_all ? 0 : (p_direct ? (int)nx : (int)nx + np);
      if (use_ortho) {
        if ((rc = ortho_drop(h, Wp, Wbase, nw, (int)nx, np, tau_ortho, !hl))) return rc;
      }
      // the explicit Rayleigh-Ritz runs the Cholesky branch on the computed
      // S^T B S even after the switch to orthogonalisation
      const bool chol_branch = !hl && (!use_ortho || direct_all);
      if ((rc = project(!chol_branch, c0, !hl))) return rc;
      int ns = (int)nx + np + nw;
      bool flip = false;
      double condR = 1.0;
      int npn = 0;
      {
        Scoped sd(h->timer, PH_DENSE);
        if (hl) {
          rc = rr_hl(h->dense, h->SAS, ns, (int)nx, (int)nc, h->Cm, &npn, h->theta, h->PAPn);
        } else {
          rc = rr_modified(h->dense, h->SAS, h->SBS, ns, (int)nx, np, (int)nc, !chol_branch,
                           tau_skip, &flip, &condR, h->Cm, &npn, h->theta, h->PAPn,
                           c0 == (int)nx + np);
        }
        if (rc) return rc;
      }
      bool chol_used = chol_branch && !flip;
      if (flip) {
        Scoped sd(h->timer, PH_DENSE);
        if (!use_ortho) {
          // Algorithm 8: switch to orthogonalisation, redo basis selection and projection
          use_ortho = true;
          h->stats.flip_iteration = it;
          if ((rc = ortho_drop(h, Wp, Wbase, nw, (int)nx, np, tau_ortho))) return rc;
          if ((rc = project(true, c0, false))) return rc;
          ns = (int)nx + np + nw;
        }
        if ((rc = rr_modified(h->dense, h->SAS, h->SBS, ns, (int)nx, np, (int)nc, true, tau_skip,
                              &flip, &condR, h->Cm, &npn, h->theta, h->PAPn, c0 == (int)nx + np)))
          return rc;
        chol_used = false;
      }
      // Algorithm 8 update and Sec. 5.2: [X, P] = S [C_x, C_p] (+ implicit products)
      const int mo = (int)nx + npn;
      const bool refresh = refresh_next || (it % refresh_every == 0);
      explicit_next = erx && refresh && !hl;
      const int* bal = h->zexp;
      if (chol_used) {
        if ((rc = diag_exponents(h->st, ns, h->SBS, ns, h->cexp))) return rc;
        bal = h->cexp;
      }
      {
        Scoped sc(h->timer, PH_UPDATE);
        SegList S = seg_empty();
        seg_push(S, h->X, ld, (int)nx);
        seg_push(S, h->P, ld, np);
        seg_push(S, Wp, ld, nw);
        OutList O{{h->Xn, h->Pn}, {ld, ld}, (int)nx};
        if ((rc = update(h, S, h->Cm, ns, mo, 1.0, 0.0, seg_empty(), O, bal))) return rc;
        if (implicit && !refresh) {
          SegList AS = seg_empty();
          seg_push(AS, h->AX, ld, (int)nx);
          seg_push(AS, h->AP, ld, np);
          seg_push(AS, h->AW, ld, nw);
          OutList AO{{h->AXn, h->APn}, {ld, ld}, (int)nx};
          if ((rc = update(h, AS, h->Cm, ns, mo, 1.0, 0.0, seg_empty(), AO, bal))) return rc;
          if (h->b_kind == 2) {
            SegList BS = seg_empty();
            seg_push(BS, h->BX, ld, (int)nx);
            seg_push(BS, h->BP, ld, np);
            seg_push(BS, h->BW, ld, nw);
            OutList BO{{h->BXn, h->BPn}, {ld, ld}, (int)nx};
            if ((rc = update(h, BS, h->Cm, ns, mo, 1.0, 0.0, seg_empty(), BO, bal))) return rc;
          }
        }
      }
      if (h->opt.inject_wait_timeout_at > 0 && it == h->opt.inject_wait_timeout_at)
        LOB_CUDA_OK(cudaMemsetAsync(h->dstatus, 1, 1, h->st));  // bit 0, as a timed-out wait
      if (!(implicit && !refresh)) {
        if ((rc = apply_AB(h, h->Xn, (int)nx, h->AXn, h->b_kind ? h->BXn : nullptr))) return rc;
        if ((rc = apply_AB(h, h->Pn, npn, h->APn, h->b_kind ? h->BPn : nullptr))) return rc;
      } else if (h->b_kind == 1) {
        if ((rc = apply_B(h, h->Xn, (int)nx, h->BXn))) return rc;
        if ((rc = apply_B(h, h->Pn, npn, h->BPn))) return rc;
      }
      std::swap(h->X, h->Xn);
      std::swap(h->P, h->Pn);
      std::swap(h->AX, h->AXn);
      std::swap(h->AP, h->APn);
      std::swap(h->BX, h->BXn);
      std::swap(h->BP, h->BPn);
      std::swap(h->PAP, h->PAPn);
      np = npn;
      // Algorithm 8: residual, preconditioned W and the convergence test
      Wbase = (Wbase == h->wbuf[0]) ? h->wbuf[1] : h->wbuf[0];
      if ((rc = residual_step(nc, true))) return rc;
      if ((rc = read_be(h, be_h.data(), nx - nc))) return rc;
      const int64_t ncn = std::max(nc, nc + leading_converged(be_h.data(), nx - nc, tol));
      refresh_next = ncn > nc;
      // Stall guard of the emulated forms: when over kStallWindow iterations
      // no column converges and the leading unconverged backward error has
      // not dropped by 10 %, the contractions have reached their accuracy
      // floor for this spectrum; the rest of the solve runs with 7 slices
      // (2^-52 per operand block) and the implicit products are refreshed.
      if (gemm_mode(h) && h->slice_boost == 0 && slices(h) < 7) {
        if (ncn != stall_nc || it - stall_it >= kStallWindow) {
          if (ncn == stall_nc && !(be_h[0] < 0.9 * stall_be) && it - stall_it >= kStallWindow) {
            h->slice_boost = 7;
            h->stats.slice_escalation_iteration = it;
            refresh_next = true;
          }
          stall_nc = ncn;
          stall_it = it;
          stall_be = be_h[std::min<int64_t>(ncn - nc, nx - nc - 1)];  // leading unconverged
        }
      }
      if ((rc = finish_w(nc, ncn))) return h->fail(rc, "preconditioner callback failed");
      nc = ncn;
    }
    if (status != LOBPCG_OK || h->opt.certify == 1) break;
    // exit certification: explicit products and Eq. (9) again
    if ((rc = apply_AB(h, h->X, (int)nx, h->AX, h->BX))) return rc;
    if ((rc = residual_step(0, false))) return rc;
    if ((rc = read_be(h, be_h.data(), nx))) return rc;
    const int64_t good = leading_converged(be_h.data(), nx, tol);
    if (good >= k) break;
    nc = good;
    refresh_next = true;
    Wbase = h->wbuf[0];
    if ((rc = residual_step(nc, true))) return rc;
    if ((rc = finish_w(nc, nc))) return h->fail(rc, "preconditioner callback failed");
  }
  if (status != LOBPCG_OK) {
    // outputs still hold the current iterate with explicit backward errors
    if ((rc = apply_AB(h, h->X, (int)nx, h->AX, h->BX))) return rc;
    if ((rc = residual_step(0, false))) return rc;
  }
  // ---- ||X^T B X - I||_F of the returned columns from explicit FP64 products
  {
    const double* bx = h->X;
    if (h->b_kind) {
      if ((rc = apply_B(h, h->X, (int)k, h->BW))) return rc;
      bx = h->BW;
    }
    if ((rc = gram_f64(h->st, n, seg1(h->X, ld, (int)k), seg1(bx, ld, (int)k), h->Gs, k, h->gwork,
                       h->gwork_bytes)))
      return rc;
    double st3[3];
    if ((rc = small_stats(h->dense, h->Gs, (int)k, (int)k, (int)k, true, h->colA, 0, h->colA, 0,
                          st3)))
      return rc;
    h->stats.orth_error = st3[0];
  }
  // ---- outputs
  if ((rc = sign_normalise(h->st, n, (int)k, h->X, ld, nullptr))) return rc;
  const cudaMemcpyKind kind =
      mem_out == LOBPCG_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  LOB_CUDA_OK(cudaMemcpy2DAsync(Xout, ldx * sizeof(double), h->X, ld * sizeof(double),
                                k * sizeof(double), n, kind, h->st));
  LOB_CUDA_OK(cudaMemcpyAsync(lambda, h->theta, k * sizeof(double), kind, h->st));
  if (resnorm) LOB_CUDA_OK(cudaMemcpyAsync(resnorm, h->be, k * sizeof(double), kind, h->st));
  h->timer.mark();
  if ((rc = to_host(h, be_h.data(), h->be, nx))) return rc;
  LOB_CUDA_OK(cudaStreamSynchronize(h->st));
  h->timer.flush();
  double mx = 0.0;
  for (int64_t i = 0; i < k; ++i) mx = std::max(mx, be_h[i]);
  h->stats.max_backward_error = mx;
  h->stats.iterations = it;
  h->stats.converged = nc;
  h->stats.gpu_launches = g_launches - launches0;
  h->stats.eig_calls = h->dense.eig_calls + h->dense.dev_calls - eig0;
  h->stats.eig_fallbacks = h->dense.eig_fallbacks + h->dense.dev_fallbacks - eigf0;
  h->stats.host_syncs = h->syncs + h->dense.syncs - syncs0;
  h->stats.eig_check_orthogonality = h->dense.check_fail[0] - cf0[0];
  h->stats.eig_check_wide_cluster = h->dense.check_fail[1] - cf0[1];
  h->stats.eig_check_nonfinite = h->dense.check_fail[2] - cf0[2];
  h->stats.ms_spmm = h->timer.total[PH_SPMM];
  h->stats.ms_gram = h->timer.total[PH_GRAM];
  h->stats.ms_update = h->timer.total[PH_UPDATE];
  h->stats.ms_residual = h->timer.total[PH_RESID];
  h->stats.ms_small_dense = h->timer.total[PH_DENSE];
  h->stats.ms_ortho = h->timer.total[PH_ORTHO];
  h->stats.ms_other = h->timer.total[PH_OTHER];
  h->stats.ms_total =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (iters) *iters = it;
  if (status == LOBPCG_ERR_NOT_CONVERGED) return h->fail(status, "maxit reached");
  if (status == LOBPCG_ERR_TIMEOUT) return h->fail(status, "wall-clock limit reached");
  return LOBPCG_OK;
}

__global__ void csr_diag_kernel(int64_t n, const int32_t* rp, const int32_t* ci, const double* v,
                                double* d) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double x = 0.0;
  for (int p = rp[r]; p < rp[r + 1]; ++p)
    if (ci[p] == r) x += v[p];
  d[r] = x;
}

int copy_in(lobpcg_ctx* h, void** dst, const void* src, size_t bytes, int mem) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  if (cudaMalloc(dst, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    return LOBPCG_ERR_OOM;
  }
  LOB_CUDA_OK(cudaMemcpyAsync(*dst, src, bytes,
                              mem == LOBPCG_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice,
                              h->st));
  return LOBPCG_OK;
}


// ---- eigenpair adjoint: dL/dA, dL/dB from (lambda, X) and dL/dlambda, dL/dX
// (first-order perturbation theory; see adjoint.cu for the formulas).
struct DevBuffers {
  std::vector<void*> p;
  ~DevBuffers() {
    for (void* q : p) cudaFree(q);
  }
  int get(void** out, size_t bytes) {
    if (cudaMalloc(out, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      return LOBPCG_ERR_OOM;
    }
    p.push_back(*out);
    return LOBPCG_OK;
  }
};

int adjoint_impl(lobpcg_ctx* h, int64_t k64, const double* lambda, const double* Xin,
                 int64_t ldx, const double* glam, const double* Gin, int64_t ldg, int mem_in,
                 double* gA, double* gB, int mem_out, double cg_tol, int cg_maxit,
                 int64_t* cg_iters) {
  const int64_t n = h->n;
  if (n <= 0) return h->fail(LOBPCG_ERR_ARG, "no operator set");
  if (k64 <= 0 || k64 > n || k64 > 2048)
    return h->fail(LOBPCG_ERR_ARG, "k must be in 1..min(n, 2048)");
  if (!lambda || !Xin || ldx < k64 || !gA) return h->fail(LOBPCG_ERR_ARG, "bad arguments");
  if (Gin && ldg < k64) return h->fail(LOBPCG_ERR_ARG, "ldg < k");
  if (h->b_kind != 0 && !gB) return h->fail(LOBPCG_ERR_ARG, "gB is needed when B is not I");
  for (int m : {mem_in, mem_out})
    if (m != LOBPCG_MEM_HOST && m != LOBPCG_MEM_DEVICE)
      return h->fail(LOBPCG_ERR_ARG, "memory kinds must be LOBPCG_MEM_HOST or LOBPCG_MEM_DEVICE");
  if (h->k_kind == 3 && !h->cb) return h->fail(LOBPCG_ERR_ARG, "no callback set");
  const int k = (int)k64;
  if (!(cg_tol > 0)) cg_tol = 1e-10;
  if (cg_maxit <= 0) cg_maxit = 20000;
  // the Gram / update scratch of the solver covers every k x k contraction
  const int64_t nx = std::max<int64_t>(h->ws_nx > 0 ? h->ws_nx : 0, k64);
  int rc = ensure_workspace(h, nx);
  if (rc) return h->fail(rc, "workspace allocation failed");
  const lobpcg_stats_t saved = h->stats;
  h->timer.st = h->st;
  h->timer.reset();
  cudaStream_t st = h->st;
  const cudaMemcpyKind kin =
      mem_in == LOBPCG_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const int64_t ld = round_up(k64, 8);
  const size_t blk = (size_t)n * ld * sizeof(double), kk = (size_t)k * k * sizeof(double),
               kv = (size_t)k * sizeof(double);
  DevBuffers D;
  double *X, *BX, *F, *Z, *P, *Q, *V, *W, *BP = nullptr;
  double *M, *Cin, *Gz, *lam, *gl, *rz0, *rz1, *pq, *rr, *caA, *cwA, *caB, *cwB;
  double *gAd = gA, *gBd = gB;
  int* flag;
  void* partial;
  for (double** b : {&X, &F, &Z, &P, &Q, &V, &W})
    if ((rc = D.get((void**)b, blk))) return h->fail(rc, "allocation failed");
  BX = X;
  if (h->b_kind != 0 && (rc = D.get((void**)&BX, blk))) return h->fail(rc, "allocation failed");
  if (h->b_kind == 2 && (rc = D.get((void**)&BP, blk))) return h->fail(rc, "allocation failed");
  for (double** b : {&M, &Cin, &Gz})
    if ((rc = D.get((void**)b, kk))) return h->fail(rc, "allocation failed");
  for (double** b : {&lam, &gl, &rz0, &rz1, &pq, &rr, &caA, &cwA, &caB, &cwB})
    if ((rc = D.get((void**)b, kv))) return h->fail(rc, "allocation failed");
  if ((rc = D.get((void**)&flag, sizeof(int))) ||
      (rc = D.get(&partial, (size_t)adj_reduce_workspace(k))))
    return h->fail(rc, "allocation failed");
  if (mem_out != LOBPCG_MEM_DEVICE) {
    if ((rc = D.get((void**)&gAd, (size_t)h->A_nnz * sizeof(double))))
      return h->fail(rc, "allocation failed");
    if (h->b_kind && (rc = D.get((void**)&gBd, (size_t)(h->b_kind == 2 ? h->B_nnz : n) *
                                                   sizeof(double))))
      return h->fail(rc, "allocation failed");
  }
  // inputs
  LOB_CUDA_OK(cudaMemcpy2DAsync(X, ld * sizeof(double), Xin, ldx * sizeof(double), kv, n, kin, st));
  LOB_CUDA_OK(cudaMemcpyAsync(lam, lambda, kv, kin, st));
  if (glam)
    LOB_CUDA_OK(cudaMemcpyAsync(gl, glam, kv, kin, st));
  else
    LOB_CUDA_OK(cudaMemsetAsync(gl, 0, kv, st));
  if (Gin)
    LOB_CUDA_OK(cudaMemcpy2DAsync(F, ld * sizeof(double), Gin, ldg * sizeof(double), kv, n, kin,
                                  st));
  else
    LOB_CUDA_OK(cudaMemsetAsync(F, 0, blk, st));
  LOB_CUDA_OK(cudaMemsetAsync(flag, 0, sizeof(int), st));
  if (h->b_kind == 1 && (rc = diag_scale(st, n, k, h->b_diag, X, ld, BX, ld))) return rc;
  if (h->b_kind == 2 &&
      (rc = spmm(st, n, h->B_rp, h->B_ci, h->B_v, X, ld, k, BX, ld, nullptr, nullptr, 0)))
    return rc;
  const SegList sX = seg1(X, ld, k), sBX = seg1(BX, ld, k), sF = seg1(F, ld, k),
                sZ = seg1(Z, ld, k), sV = seg1(V, ld, k);
  // M = X^T G (g_i^T x_i on its diagonal)
  if ((rc = gram(h, sX, sF, M, k))) return rc;
  if ((rc = grad_coeff(st, k, lam, gl, M, k, caA, cwA, caB, cwB))) return rc;
  int64_t its = 0;
  bool converged = true;
  if (Gin) {
    std::vector<double> lh(k);
    if ((rc = to_host(h, lh.data(), lam, k))) return rc;
    double scale = h->stats.norm_a;
    for (double x : lh) scale = std::max(scale, std::fabs(x));
    if ((rc = adj_coeff(st, k, M, k, lam, 1e-10 * scale, Cin, flag))) return rc;
    // F = (I - B X X^T) G
    if ((rc = update(h, sBX, M, k, k, -1.0, 1.0, sF, out1(F, ld, k), h->zexp))) return rc;
    std::vector<double> f2(k), r2(k);
    if ((rc = colsumsq(st, n, F, ld, k, rr, h->rwork))) return rc;
    if ((rc = to_host(h, f2.data(), rr, k))) return rc;
    int fl = 0;
    LOB_CUDA_OK(cudaMemcpyAsync(h->hbuf, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LOB_CUDA_OK(cudaStreamSynchronize(st));
    memcpy(&fl, h->hbuf, sizeof(int));
    if (fl) {
      h->stats = saved;
      return h->fail(LOBPCG_ERR_DEGENERATE,
                     "two wanted eigenvalues are closer than 1e-10 max(|lambda|, ||A||)");
    }
    const double* kd = (h->k_kind == 0) ? h->adiag : (h->k_kind == 1 ? h->kdiag : nullptr);
    if (kd) {  // cg_step applies K^-1 as a product with the reciprocal
      if ((rc = reciprocal(st, n, kd, h->kinv))) return rc;
      kd = h->kinv;
    }
    // project Z onto the B-orthogonal complement of X: Z -= X (BX^T Z)
    auto project = [&]() -> int {
      int r;
      if ((r = gram(h, sBX, sZ, Gz, k))) return r;
      return update(h, sX, Gz, k, k, -1.0, 1.0, sZ, out1(Z, ld, k), h->zexp);
    };
    auto precond = [&]() -> int {
      if (h->k_kind != 3) return LOBPCG_OK;  // Z = R / kdiag was written by cg_step
      return h->cb(h->cb_ctx, n, k, F, ld, Z, ld, (void*)st) ? LOBPCG_ERR_CALLBACK : LOBPCG_OK;
    };
    // u_0 = 0 (V = -u), R = F; Z = P_B K^-1 R; P = Z
    LOB_CUDA_OK(cudaMemsetAsync(V, 0, blk, st));
    LOB_CUDA_OK(cudaMemsetAsync(pq, 0, kv, st));
    if ((rc = cg_step(st, n, k, V, V, F, F, Z, kd, ld, pq, pq, rr, partial))) return rc;
    if ((rc = precond())) return h->fail(rc, "preconditioner callback failed");
    if ((rc = project())) return rc;
    if ((rc = coldot(st, n, k, F, Z, ld, rz0, partial))) return rc;
    if ((rc = copy_block(st, n, k, Z, ld, P, ld))) return rc;
    converged = false;
    for (int64_t it = 1; it <= cg_maxit; ++it) {
      if ((rc = spmm(st, n, h->A_rp, h->A_ci, h->A_v, P, ld, k, Q, ld, nullptr, nullptr, 0)))
        return rc;
      if (h->b_kind == 2 &&
          (rc = spmm(st, n, h->B_rp, h->B_ci, h->B_v, P, ld, k, BP, ld, nullptr, nullptr, 0)))
        return rc;
      if ((rc = shift_dot(st, n, k, Q, P, BP, h->b_kind == 1 ? h->b_diag : nullptr, ld, lam, pq,
                          partial)))
        return rc;
      if ((rc = cg_step(st, n, k, V, P, F, Q, Z, kd, ld, rz0, pq, rr, partial))) return rc;
      if ((rc = precond())) return h->fail(rc, "preconditioner callback failed");
      if ((rc = project())) return rc;
      if ((rc = coldot(st, n, k, F, Z, ld, rz1, partial))) return rc;
      if ((rc = cg_direction(st, n, k, P, Z, ld, rz1, rz0))) return rc;
      std::swap(rz0, rz1);
      its = it;
      if (it % 8 == 0 || it == cg_maxit) {
        if ((rc = to_host(h, r2.data(), rr, k))) return rc;
        bool all = true;
        for (int j = 0; j < k; ++j) all = all && !(r2[j] > cg_tol * cg_tol * f2[j]);
        if (all) {
          converged = true;
          break;
        }
      }
    }
    // W = X Cin - u
    if ((rc = update(h, sX, Cin, k, k, 1.0, 1.0, sV, out1(W, ld, k), h->zexp))) return rc;
  } else {
    LOB_CUDA_OK(cudaMemsetAsync(W, 0, blk, st));
  }
  if ((rc = pattern_grad(st, n, h->A_rp, h->A_ci, X, W, ld, k, caA, cwA, gAd))) return rc;
  if (h->b_kind == 1 && (rc = diag_grad(st, n, X, W, ld, k, caB, cwB, gBd))) return rc;
  if (h->b_kind == 2 &&
      (rc = pattern_grad(st, n, h->B_rp, h->B_ci, X, W, ld, k, caB, cwB, gBd)))
    return rc;
  if (mem_out != LOBPCG_MEM_DEVICE) {
    LOB_CUDA_OK(cudaMemcpyAsync(gA, gAd, (size_t)h->A_nnz * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
    if (h->b_kind)
      LOB_CUDA_OK(cudaMemcpyAsync(gB, gBd,
                                  (size_t)(h->b_kind == 2 ? h->B_nnz : n) * sizeof(double),
                                  cudaMemcpyDeviceToHost, st));
  }
  LOB_CUDA_OK(cudaStreamSynchronize(st));
  h->timer.flush();
  h->stats = saved;
  if (cg_iters) *cg_iters = its;
  if (!converged)
    return h->fail(LOBPCG_ERR_NOT_CONVERGED, "adjoint CG reached cg_maxit (outputs written)");
  return LOBPCG_OK;
}

}  // namespace

// ============================================================== C ABI

LOBPCG_EXPORT int lobpcg_create(lobpcg_t* out, const lobpcg_options_t* opts, void* stream) {
  if (!out) return LOBPCG_ERR_ARG;
  *out = nullptr;
  auto* h = new (std::nothrow) lobpcg_ctx();
  if (!h) return LOBPCG_ERR_OOM;
  if (opts) h->opt = *opts;
  if (h->opt.gemm_mode != LOBPCG_GEMM_F64 && h->opt.gemm_mode != LOBPCG_GEMM_OZAKI &&
      h->opt.gemm_mode != LOBPCG_GEMM_OZAKI_TC) {
    delete h;
    return LOBPCG_ERR_ARG;
  }
  if (h->opt.ozaki_slices != 0 && (h->opt.ozaki_slices < 3 || h->opt.ozaki_slices > 7)) {
    delete h;
    return LOBPCG_ERR_ARG;
  }
  cudaGetDevice(&h->device);
  h->st = (cudaStream_t)stream;
  if (cudaMallocHost(&h->hbuf, 1 << 20) != cudaSuccess) {
    delete h;
    return LOBPCG_ERR_OOM;
  }
  *out = h;
  return LOBPCG_OK;
}

LOBPCG_EXPORT void lobpcg_destroy(lobpcg_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  delete h;
}

LOBPCG_EXPORT const char* lobpcg_last_error(lobpcg_t h) { return h ? h->err.c_str() : "null handle"; }

LOBPCG_EXPORT int lobpcg_get_stats(lobpcg_t h, lobpcg_stats_t* out) {
  if (!h || !out) return LOBPCG_ERR_ARG;
  *out = h->stats;
  return LOBPCG_OK;
}

namespace {

__global__ void widen_kernel(int64_t count, const float* __restrict__ src, double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = (double)src[i];
}

// value array of the operator into the handle: FP64 copied (or used in place
// when borrowed), FP32 widened to FP64 (on the host for host arrays, by a
// kernel for device arrays)
int values_in(lobpcg_ctx* h, double** dst, const void* src, int64_t count, int dtype, int mem,
              bool borrow, unsigned bit) {
  if (dtype == LOBPCG_F64) {
    if (borrow) {
      *dst = static_cast<double*>(const_cast<void*>(src));
      h->borrowed |= 1u << bit;
      return LOBPCG_OK;
    }
    return copy_in(h, (void**)dst, src, (size_t)count * sizeof(double), mem);
  }
  if (mem == LOBPCG_MEM_HOST) {
    const float* f = static_cast<const float*>(src);
    std::vector<double> w(f, f + count);
    return copy_in(h, (void**)dst, w.data(), (size_t)count * sizeof(double), LOBPCG_MEM_HOST);
  }
  if (cudaMalloc((void**)dst, std::max<size_t>((size_t)count * sizeof(double), 16)) !=
      cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    return LOBPCG_ERR_OOM;
  }
  if (count > 0) {
    widen_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, h->st>>>(
        count, static_cast<const float*>(src), *dst);
    ++g_launches;
    if (cudaPeekAtLastError() != cudaSuccess) return LOBPCG_ERR_CUDA;
  }
  return LOBPCG_OK;
}

int index_in(lobpcg_ctx* h, int32_t** dst, const int32_t* src, int64_t count, int mem,
             bool borrow, unsigned bit) {
  if (borrow) {
    *dst = const_cast<int32_t*>(src);
    h->borrowed |= 1u << bit;
    return LOBPCG_OK;
  }
  return copy_in(h, (void**)dst, src, (size_t)count * sizeof(int32_t), mem);
}

int set_operator_impl(lobpcg_t h, int64_t n, const int32_t* A_rowptr, const int32_t* A_col,
                      const void* A_val, int64_t A_nnz, int A_dtype, const int32_t* B_rowptr,
                      const int32_t* B_col, const void* B_val, int64_t B_nnz,
                      const void* B_diag, int B_dtype, int mem, int flags) {
  if (!h) return LOBPCG_ERR_ARG;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return h->fail(LOBPCG_ERR_ARG, "handle belongs to another device");
  // Any other failure leaves the handle without an operator, so that a later solve
  // or adjoint returns LOBPCG_ERR_ARG instead of using stale, freed or
  // partial buffers.
  auto drop = [h](int code, const char* msg) {
    h->free_ws();
    h->release_op();
    h->n = h->A_nnz = h->B_nnz = 0;
    h->b_kind = 0;
    h->b_cond = 1.0;
    h->k_kind = 0;
    return h->fail(code, msg);
  };
  if (n <= 0 || n > (int64_t)1 << 31) return drop(LOBPCG_ERR_ARG, "n out of range");
  if (!A_rowptr || !A_col || !A_val || A_nnz < 0 || A_nnz >= ((int64_t)1 << 31))
    return drop(LOBPCG_ERR_ARG, "bad A");
  if (B_rowptr && (!B_col || !B_val || B_nnz < 0 || B_nnz >= ((int64_t)1 << 31)))
    return drop(LOBPCG_ERR_ARG, "bad B");
  if (B_rowptr && B_diag) return drop(LOBPCG_ERR_ARG, "give B as CSR or diagonal, not both");
  if ((A_dtype != LOBPCG_F64 && A_dtype != LOBPCG_F32) ||
      (B_dtype != LOBPCG_F64 && B_dtype != LOBPCG_F32))
    return drop(LOBPCG_ERR_ARG, "value dtype must be LOBPCG_F64 or LOBPCG_F32");
  if ((flags & ~LOBPCG_BORROW) != 0) return drop(LOBPCG_ERR_ARG, "unknown flags");
  const bool borrow = (flags & LOBPCG_BORROW) != 0;
  if (borrow && mem != LOBPCG_MEM_DEVICE)
    return drop(LOBPCG_ERR_ARG, "only device arrays can be borrowed");
  if (mem == LOBPCG_MEM_HOST) {
    // host arrays are checked before anything is copied: the kernels index
    // through rowptr and col without bounds checks
    auto csr_ok = [n](const int32_t* rp, const int32_t* ci, int64_t nnz) {
      if (rp[0] != 0 || rp[n] != nnz) return false;
      for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return false;
      for (int64_t p = 0; p < nnz; ++p)
        if (ci[p] < 0 || ci[p] >= n) return false;
      return true;
    };
    if (!csr_ok(A_rowptr, A_col, A_nnz)) return drop(LOBPCG_ERR_ARG, "A is not a valid n x n CSR");
    if (B_rowptr && !csr_ok(B_rowptr, B_col, B_nnz))
      return drop(LOBPCG_ERR_ARG, "B is not a valid n x n CSR");
    if (B_diag)
      for (int64_t i = 0; i < n; ++i) {
        const double b = B_dtype == LOBPCG_F32 ? (double)static_cast<const float*>(B_diag)[i]
                                               : static_cast<const double*>(B_diag)[i];
        if (!(b > 0)) return drop(LOBPCG_ERR_ARG, "diagonal B must be positive");
      }
  } else if (mem != LOBPCG_MEM_DEVICE) {
    return drop(LOBPCG_ERR_ARG, "mem must be LOBPCG_MEM_HOST or LOBPCG_MEM_DEVICE");
  }
  h->free_ws();
  h->release_op();
  h->n = n;
  h->A_nnz = A_nnz;
  int rc;
  if ((rc = index_in(h, &h->A_rp, A_rowptr, n + 1, mem, borrow, 0)) ||
      (rc = index_in(h, &h->A_ci, A_col, A_nnz, mem, borrow, 1)) ||
      (rc = values_in(h, &h->A_v, A_val, A_nnz, A_dtype, mem, borrow, 2)))
    return drop(rc, "copying A failed");
  h->b_kind = 0;
  h->b_cond = 1.0;
  if (B_rowptr) {
    h->b_kind = 2;
    h->B_nnz = B_nnz;
    if ((rc = index_in(h, &h->B_rp, B_rowptr, n + 1, mem, borrow, 3)) ||
        (rc = index_in(h, &h->B_ci, B_col, B_nnz, mem, borrow, 4)) ||
        (rc = values_in(h, &h->B_v, B_val, B_nnz, B_dtype, mem, borrow, 5)))
      return drop(rc, "copying B failed");
  } else if (B_diag) {
    h->b_kind = 1;
    // the diagonal is always copied into the handle (FP64), never borrowed
    if ((rc = values_in(h, &h->b_diag, B_diag, n, B_dtype, mem, false, 6)))
      return drop(rc, "copying B failed");
    std::vector<double> b(n);
    if (cudaMemcpyAsync(b.data(), h->b_diag, n * sizeof(double), cudaMemcpyDeviceToHost, h->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess)
      return drop(LOBPCG_ERR_CUDA, "reading B failed");
    double lo = INFINITY, hi = 0.0;
    for (double x : b) {
      lo = std::min(lo, std::fabs(x));
      hi = std::max(hi, std::fabs(x));
      if (!(x > 0)) return drop(LOBPCG_ERR_ARG, "diagonal B must be positive");
    }
    h->b_cond = hi / lo;
  }
  if (cudaMalloc(&h->adiag, n * sizeof(double)) != cudaSuccess) {
    h->adiag = nullptr;
    return drop(LOBPCG_ERR_OOM, "allocation failed");
  }
  csr_diag_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, h->st>>>(n, h->A_rp, h->A_ci, h->A_v,
                                                                 h->adiag);
  ++g_launches;
  std::vector<double> d(n);
  if (cudaMemcpyAsync(d.data(), h->adiag, n * sizeof(double), cudaMemcpyDeviceToHost, h->st) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess)
    return drop(LOBPCG_ERR_CUDA, "reading diag(A) failed");
  h->k_kind = 0;
  for (double x : d)
    if (x == 0.0) {
      h->k_kind = 2;  // Jacobi undefined: fall back to K = I and report it
      h->err = "diag(A) has a zero entry: preconditioner set to K = I";
      break;
    }
  return LOBPCG_OK;
}

}  // namespace

LOBPCG_EXPORT int lobpcg_set_operator(lobpcg_t h, int64_t n, const int32_t* A_rowptr,
                                      const int32_t* A_col, const double* A_val, int64_t A_nnz,
                                      const int32_t* B_rowptr, const int32_t* B_col,
                                      const double* B_val, int64_t B_nnz, const double* B_diag,
                                      int mem) {
  return set_operator_impl(h, n, A_rowptr, A_col, A_val, A_nnz, LOBPCG_F64, B_rowptr, B_col,
                           B_val, B_nnz, B_diag, LOBPCG_F64, mem, 0);
}

LOBPCG_EXPORT int lobpcg_set_operator_ex(lobpcg_t h, int64_t n, const int32_t* A_rowptr,
                                         const int32_t* A_col, const void* A_val, int64_t A_nnz,
                                         int A_dtype, const int32_t* B_rowptr,
                                         const int32_t* B_col, const void* B_val, int64_t B_nnz,
                                         const void* B_diag, int B_dtype, int mem, int flags) {
  return set_operator_impl(h, n, A_rowptr, A_col, A_val, A_nnz, A_dtype, B_rowptr, B_col, B_val,
                           B_nnz, B_diag, B_dtype, mem, flags);
}

LOBPCG_EXPORT int lobpcg_set_precond_diag(lobpcg_t h, const double* kdiag, int mem) {
  if (!h) return LOBPCG_ERR_ARG;
  if (h->n <= 0) return h->fail(LOBPCG_ERR_ARG, "set the operator first");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return h->fail(LOBPCG_ERR_ARG, "handle belongs to another device");
  if (mem < 0) {
    h->k_kind = 2;
    return LOBPCG_OK;
  }
  if (!kdiag) {
    h->k_kind = 0;
    return LOBPCG_OK;
  }
  if (mem != LOBPCG_MEM_HOST && mem != LOBPCG_MEM_DEVICE)
    return h->fail(LOBPCG_ERR_ARG, "mem must be negative, LOBPCG_MEM_HOST or LOBPCG_MEM_DEVICE");
  if (mem == LOBPCG_MEM_HOST)
    for (int64_t i = 0; i < h->n; ++i)
      if (!(kdiag[i] > 0)) return h->fail(LOBPCG_ERR_ARG, "diagonal K must be positive");
  int rc = copy_in(h, (void**)&h->kdiag, kdiag, h->n * sizeof(double), mem);
  if (rc) {
    h->k_kind = 0;
    return h->fail(rc, "copying K failed");
  }
  h->k_kind = 1;
  return LOBPCG_OK;
}

LOBPCG_EXPORT int lobpcg_set_precond_callback(lobpcg_t h, lobpcg_precond_fn fn, void* ctx) {
  if (!h || !fn) return LOBPCG_ERR_ARG;
  h->cb = fn;
  h->cb_ctx = ctx;
  h->k_kind = 3;
  return LOBPCG_OK;
}

LOBPCG_EXPORT int lobpcg_solve(lobpcg_t h, int64_t k, double tol, const double* X0,
                               int64_t ldx0, uint64_t seed, int mem_in, double* lambda,
                               double* X, int64_t ldx, int mem_out, int64_t* iters,
                               double* resnorm) {
  if (!h) return LOBPCG_ERR_ARG;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return h->fail(LOBPCG_ERR_ARG, "handle belongs to another device");
  h->err.clear();
  h->stats.iterations = 0;
  int rc = solve_impl(h, k, tol, X0, ldx0, seed, mem_in, lambda, X, ldx, mem_out, iters, resnorm);
  if (rc && rc != LOBPCG_ERR_NOT_CONVERGED && iters) *iters = h->stats.iterations;
  if (rc == LOBPCG_ERR_CUDA && h->err.empty()) {
    cudaError_t e = cudaGetLastError();
    h->err = std::string("CUDA error: ") + cudaGetErrorString(e);
  } else if (rc && h->err.empty()) {
    h->err = "solve failed";
  }
  return rc;
}

LOBPCG_EXPORT int lobpcg_eig_adjoint(lobpcg_t h, int64_t k, const double* lambda, const double* X,
                                     int64_t ldx, const double* glam, const double* G,
                                     int64_t ldg, int mem_in, double* gA, double* gB,
                                     int mem_out, double cg_tol, int32_t cg_maxit,
                                     int64_t* cg_iters) {
  if (!h) return LOBPCG_ERR_ARG;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return h->fail(LOBPCG_ERR_ARG, "handle belongs to another device");
  h->err.clear();
  int rc = adjoint_impl(h, k, lambda, X, ldx, glam, G, ldg, mem_in, gA, gB, mem_out, cg_tol,
                        cg_maxit, cg_iters);
  if (rc == LOBPCG_ERR_CUDA && h->err.empty()) {
    cudaError_t e = cudaGetLastError();
    h->err = std::string("CUDA error: ") + cudaGetErrorString(e);
  } else if (rc && h->err.empty()) {
    h->err = "adjoint failed";
  }
  return rc;
}
