"""ctypes binding of the C ABI declared in include/lobpcg.h (argument marshalling only).

Every function here forwards to the shared library built by build.py; nothing
computes on the host.  Loading fails loudly when the library is missing.
"""
import ctypes
import os

from . import build as _build

LOBPCG_OK = 0
LOBPCG_ERR_ARG = 1
LOBPCG_ERR_NOT_CONVERGED = 2
LOBPCG_ERR_BREAKDOWN = 3
LOBPCG_ERR_CUDA = 4
LOBPCG_ERR_OOM = 5
LOBPCG_ERR_TIMEOUT = 6
LOBPCG_ERR_CALLBACK = 7
LOBPCG_ERR_DEGENERATE = 8

LOBPCG_MEM_HOST = 0
LOBPCG_MEM_DEVICE = 1
LOBPCG_F64 = 0
LOBPCG_F32 = 1
LOBPCG_BORROW = 1
LOBPCG_GEMM_F64 = 0
LOBPCG_GEMM_OZAKI = 1
LOBPCG_GEMM_OZAKI_TC = 2

STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_NOT_CONVERGED", 3: "ERR_BREAKDOWN",
                4: "ERR_CUDA", 5: "ERR_OOM", 6: "ERR_TIMEOUT", 7: "ERR_CALLBACK",
                8: "ERR_DEGENERATE"}

EXPORTED = [
    "lobpcg_create", "lobpcg_set_operator", "lobpcg_set_precond_diag",
    "lobpcg_set_precond_callback", "lobpcg_solve", "lobpcg_get_stats", "lobpcg_last_error",
    "lobpcg_destroy", "lobpcg_spmm", "lobpcg_gram", "lobpcg_gram_workspace",
    "lobpcg_update", "lobpcg_residual", "lobpcg_philox_normal", "lobpcg_gram_noalloc",
    "lobpcg_eig_adjoint", "lobpcg_syev",
    "lobpcg_chebyshev_create", "lobpcg_chebyshev_apply", "lobpcg_chebyshev_destroy",
    "lobpcg_wait_selftest", "lobpcg_set_operator_ex",
]


class lobpcg_options_t(ctypes.Structure):
    _fields_ = [
        ("block_width", ctypes.c_int64),
        ("maxit", ctypes.c_int32),
        ("implicit", ctypes.c_int32),
        ("refresh_every", ctypes.c_int32),
        ("omega_rows", ctypes.c_int32),
        ("gemm_mode", ctypes.c_int32),
        ("ozaki_slices", ctypes.c_int32),
        ("certify", ctypes.c_int32),
        ("tau_ortho", ctypes.c_double),
        ("tau_skip", ctypes.c_double),
        ("max_seconds", ctypes.c_double),
        ("dense_eig", ctypes.c_int32),
        ("basis", ctypes.c_int32),
        ("explicit_rr", ctypes.c_int32),
        ("criterion", ctypes.c_int32),
        ("gram_blocks", ctypes.c_int32),
        ("inject_wait_timeout_at", ctypes.c_int32),
    ]


class lobpcg_stats_t(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int64),
        ("n_x", ctypes.c_int64),
        ("converged", ctypes.c_int64),
        ("flip_iteration", ctypes.c_int64),
        ("ortho_calls", ctypes.c_int64),
        ("svqb_passes", ctypes.c_int64),
        ("dropped_columns", ctypes.c_int64),
        ("gpu_launches", ctypes.c_int64),
        ("norm_a", ctypes.c_double),
        ("norm_b", ctypes.c_double),
        ("max_backward_error", ctypes.c_double),
        ("ms_spmm", ctypes.c_double),
        ("ms_gram", ctypes.c_double),
        ("ms_update", ctypes.c_double),
        ("ms_residual", ctypes.c_double),
        ("ms_small_dense", ctypes.c_double),
        ("ms_ortho", ctypes.c_double),
        ("ms_other", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("spmm_calls", ctypes.c_int64),
        ("gram_calls", ctypes.c_int64),
        ("update_calls", ctypes.c_int64),
        ("spmm_bytes", ctypes.c_double),
        ("gram_flops", ctypes.c_double),
        ("update_flops", ctypes.c_double),
        ("gram_tensor_flops", ctypes.c_double),
        ("update_tensor_flops", ctypes.c_double),
        ("eig_calls", ctypes.c_int64),
        ("eig_fallbacks", ctypes.c_int64),
        ("slice_escalation_iteration", ctypes.c_int64),
        ("gram_bytes", ctypes.c_double),
        ("update_bytes", ctypes.c_double),
        ("orth_error", ctypes.c_double),
        ("host_syncs", ctypes.c_int64),
        ("eig_check_orthogonality", ctypes.c_int64),
        ("eig_check_wide_cluster", ctypes.c_int64),
        ("eig_check_nonfinite", ctypes.c_int64),
        ("explicit_rr_calls", ctypes.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


PRECOND_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                              ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                              ctypes.c_void_p)

_lib = None

P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int
D = ctypes.c_double


def library_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load the shared library (building it first only when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(
                f"CUDA library {path} is not built; run `python -m paper_1704_07458_gb300.build`")
        _build.build()
    lib = ctypes.CDLL(path)
    sig = {
        "lobpcg_create": (I32, [ctypes.POINTER(P), ctypes.POINTER(lobpcg_options_t), P]),
        "lobpcg_set_operator": (I32, [P, I64, P, P, P, I64, P, P, P, I64, P, I32]),
        "lobpcg_set_precond_diag": (I32, [P, P, I32]),
        "lobpcg_set_precond_callback": (I32, [P, PRECOND_FN, P]),
        "lobpcg_solve": (I32, [P, I64, D, P, I64, ctypes.c_uint64, I32, P, P, I64, I32,
                               ctypes.POINTER(I64), P]),
        "lobpcg_get_stats": (I32, [P, ctypes.POINTER(lobpcg_stats_t)]),
        "lobpcg_last_error": (ctypes.c_char_p, [P]),
        "lobpcg_destroy": (None, [P]),
        "lobpcg_spmm": (I32, [I64, P, P, P, P, I64, I64, P, I64, P, P, I64, P]),
        "lobpcg_gram": (I32, [I64, P, I64, I64, P, I64, I64, P, I64, I32, I32, P, I64, P]),
        "lobpcg_gram_workspace": (I64, [I64, I64, I64, I32, I32]),
        "lobpcg_gram_noalloc": (I32, [I64, P, I64, I64, P, I64, I64, P, I64, I32, P]),
        "lobpcg_update": (I32, [I64, P, I64, I64, P, I64, I64, D, D, P, I64, P, I64, I32, I32,
                                P]),
        "lobpcg_residual": (I32, [I64, P, P, P, I64, I64, I64, P, P, P, I64, D, D, P, P]),
        "lobpcg_philox_normal": (I32, [I64, I64, ctypes.c_uint64, ctypes.c_uint32, P, I64, P]),
        "lobpcg_syev": (I32, [I64, P, I64, P, I32, P]),
        "lobpcg_eig_adjoint": (I32, [P, I64, P, P, I64, P, P, I64, I32, P, P, I32, D, I32,
                                     ctypes.POINTER(I64)]),
        "lobpcg_chebyshev_create": (I32, [ctypes.POINTER(P), I64, P, P, P, P, I32, D, D, I64]),
        "lobpcg_chebyshev_apply": (I32, [P, I64, I64, P, I64, P, I64, P]),
        "lobpcg_chebyshev_destroy": (None, [P]),
        "lobpcg_wait_selftest": (I32, [I32, P]),
        "lobpcg_set_operator_ex": (I32, [P, I64, P, P, P, I64, I32, P, P, P, I64, P, I32, I32,
                                         I32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def ptr(x):
    """Raw address of a numpy array, a torch tensor or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return int(x)


def stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class LobpcgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code, what=""):
    if code != LOBPCG_OK:
        raise LobpcgError(code, what)
    return code


# ---- one Python function per C entry point (same names) -------------------

def lobpcg_create(opts=None, stream=None):
    lib = load()
    h = P()
    o = ctypes.byref(opts) if opts is not None else None
    check(lib.lobpcg_create(ctypes.byref(h), o, stream_ptr(stream)), "lobpcg_create")
    return h


def lobpcg_set_operator(h, n, A_rowptr, A_col, A_val, A_nnz, B_rowptr=None, B_col=None,
                        B_val=None, B_nnz=0, B_diag=None, mem=LOBPCG_MEM_HOST):
    lib = load()
    return lib.lobpcg_set_operator(h, n, ptr(A_rowptr), ptr(A_col), ptr(A_val), A_nnz,
                                   ptr(B_rowptr), ptr(B_col), ptr(B_val), B_nnz, ptr(B_diag),
                                   mem)


def lobpcg_set_operator_ex(h, n, A_rowptr, A_col, A_val, A_nnz, A_dtype=LOBPCG_F64,
                           B_rowptr=None, B_col=None, B_val=None, B_nnz=0, B_diag=None,
                           B_dtype=LOBPCG_F64, mem=LOBPCG_MEM_HOST, flags=0):
    return load().lobpcg_set_operator_ex(h, n, ptr(A_rowptr), ptr(A_col), ptr(A_val), A_nnz,
                                         A_dtype, ptr(B_rowptr), ptr(B_col), ptr(B_val), B_nnz,
                                         ptr(B_diag), B_dtype, mem, flags)


def lobpcg_set_precond_diag(h, kdiag, mem=LOBPCG_MEM_HOST):
    return load().lobpcg_set_precond_diag(h, ptr(kdiag), mem)


def lobpcg_set_precond_callback(h, fn, ctx=None):
    return load().lobpcg_set_precond_callback(h, fn, ctx)


def lobpcg_chebyshev_create(n, rowptr, col, val, diag, degree, lmin, lmax, max_cols):
    c = P()
    rc = load().lobpcg_chebyshev_create(ctypes.byref(c), n, ptr(rowptr), ptr(col), ptr(val),
                                        ptr(diag), degree, lmin, lmax, max_cols)
    check(rc, "lobpcg_chebyshev_create")
    return c


def lobpcg_chebyshev_apply(ctx, n, ncols, R, ldr, W, ldw, stream=None):
    return load().lobpcg_chebyshev_apply(ctx, n, ncols, ptr(R), ldr, ptr(W), ldw,
                                         stream_ptr(stream))


def lobpcg_chebyshev_destroy(c):
    load().lobpcg_chebyshev_destroy(c)


def chebyshev_callback():
    """lobpcg_chebyshev_apply as a callback pointer (called by the library
    itself, no Python on the path)."""
    return ctypes.cast(load().lobpcg_chebyshev_apply, PRECOND_FN)


def lobpcg_solve(h, k, tol, X0, ldx0, seed, mem_in, lam, X, ldx, mem_out, resnorm=None):
    it = I64(0)
    rc = load().lobpcg_solve(h, k, tol, ptr(X0), ldx0, seed, mem_in, ptr(lam), ptr(X), ldx,
                             mem_out, ctypes.byref(it), ptr(resnorm))
    return rc, it.value


def lobpcg_get_stats(h):
    s = lobpcg_stats_t()
    check(load().lobpcg_get_stats(h, ctypes.byref(s)), "lobpcg_get_stats")
    return s


def lobpcg_last_error(h):
    m = load().lobpcg_last_error(h)
    return m.decode() if m else ""


def lobpcg_destroy(h):
    load().lobpcg_destroy(h)


def lobpcg_spmm(n, rowptr, col, val, X, ldx, m, Y, ldy, b=None, BY=None, ldby=0, stream=None):
    return load().lobpcg_spmm(n, ptr(rowptr), ptr(col), ptr(val), ptr(X), ldx, m, ptr(Y), ldy,
                              ptr(b), ptr(BY), ldby, stream_ptr(stream))


def lobpcg_gram_workspace(n, p, q, mode=LOBPCG_GEMM_F64, slices=0):
    return load().lobpcg_gram_workspace(n, p, q, mode, slices)


def lobpcg_gram(n, U, ldu, p, V, ldv, q, G, ldg, mode=LOBPCG_GEMM_F64, slices=0, work=None,
                work_bytes=0, stream=None):
    return load().lobpcg_gram(n, ptr(U), ldu, p, ptr(V), ldv, q, ptr(G), ldg, mode, slices,
                              ptr(work), work_bytes, stream_ptr(stream))


def lobpcg_gram_noalloc(n, U, ldu, p, V, ldv, q, G, ldg, slices=0, stream=None):
    """G = U^T V without allocating (fixed in-library scratch; see lobpcg.h)."""
    return load().lobpcg_gram_noalloc(n, ptr(U), ldu, p, ptr(V), ldv, q, ptr(G), ldg, slices,
                                      stream_ptr(stream))


def lobpcg_wait_selftest(polls, stream=None):
    """Bounded-wait self-test (see lobpcg.h): LOBPCG_ERR_TIMEOUT when the wait ran out."""
    return load().lobpcg_wait_selftest(polls, stream_ptr(stream))


def lobpcg_update(n, S, lds, s, C, ldc, m, alpha, beta, Y0, ldy0, Y, ldy,
                  mode=LOBPCG_GEMM_F64, slices=0, stream=None):
    return load().lobpcg_update(n, ptr(S), lds, s, ptr(C), ldc, m, alpha, beta, ptr(Y0), ldy0,
                                ptr(Y), ldy, mode, slices, stream_ptr(stream))


def lobpcg_residual(n, X, AX, BX, ld, m, c0, theta, kdiag, W, ldw, normA, normB, be,
                    stream=None):
    return load().lobpcg_residual(n, ptr(X), ptr(AX), ptr(BX), ld, m, c0, ptr(theta),
                                  ptr(kdiag), ptr(W), ldw, normA, normB, ptr(be),
                                  stream_ptr(stream))


def lobpcg_philox_normal(n, m, seed, stream_id, Y, ldy, stream=None):
    return load().lobpcg_philox_normal(n, m, seed, stream_id, ptr(Y), ldy, stream_ptr(stream))


def lobpcg_eig_adjoint(h, k, lam, X, ldx, glam, G, ldg, mem_in, gA, gB, mem_out, cg_tol=0.0,
                       cg_maxit=0):
    """Gradients of the eigenpairs with respect to the stored values of A and B
    (see lobpcg.h).  Returns (status, CG iterations)."""
    it = I64(0)
    rc = load().lobpcg_eig_adjoint(h, k, ptr(lam), ptr(X), ldx, ptr(glam), ptr(G), ldg, mem_in,
                                   ptr(gA), ptr(gB), mem_out, cg_tol, cg_maxit, ctypes.byref(it))
    return rc, it.value


def lobpcg_syev(n, A, lda, w, mode=0, stream=None):
    """Eigendecomposition of a small symmetric matrix in place (see lobpcg.h)."""
    return load().lobpcg_syev(n, ptr(A), lda, ptr(w), mode, stream_ptr(stream))
