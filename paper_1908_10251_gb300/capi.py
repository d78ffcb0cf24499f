"""Thin ctypes binding of libpasm (include/pasm.h), one Python function per
C entry point with the same name.  Argument marshalling only: every step of
the method runs in the library's CUDA kernels.  There is no fallback: if the
shared library is missing or fails to load, every call raises.

Arrays may be numpy arrays (host memory) or torch CUDA tensors (device
memory); block vectors are n x k row-major float64, eigenvalues float64,
per-pair counters int32.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpasm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pasm.h")

PASM_OK, PASM_EINVAL, PASM_EK_TOO_BIG, PASM_ENOMEM, PASM_ECUDA = 0, 1, 2, 3, 4
PASM_ENOTCONV, PASM_EDEGENERATE, PASM_ENAN, PASM_ESTATE, PASM_ENOTPD, PASM_ETIMEOUT = 5, 6, 7, 8, 9, 10
PASM_PAIR_ACTIVE, PASM_PAIR_CONVERGED, PASM_PAIR_DEGENERATE, PASM_PAIR_NAN = 0, 1, 2, 3
PASM_FP64, PASM_MIXED = 0, 1
PASM_SCORE_A, PASM_SCORE_B = 0, 1
PASM_INIT_COARSE, PASM_INIT_NESTED = 0, 1
PASM_JACOBI, PASM_LEARNED, PASM_CG = 0, 1, 2
PASM_PROJ_TENSOR, PASM_PROJ_FP64 = 0, 1
TILE_KINDS = ("jacobi", "jacobi2_zero", "resid_restrict", "resid", "restrict", "prolong", "outer_rhs",
              "outer_res", "border", "chain_r", "chain_p", "update", "prolong_sweep", "restrict_first")
PASM_TILE_N = len(TILE_KINDS)
NN_WEIGHTS = 2592


class pasm_csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class pasm_opts(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("cycles_per_step", ctypes.c_int), ("max_steps", ctypes.c_int), ("precision", ctypes.c_int),
                ("score_norm", ctypes.c_int), ("init", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("smoother", ctypes.c_int), ("projection", ctypes.c_int), ("autotune", ctypes.c_int),
                ("res_tol", ctypes.c_double)]


class PasmError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__("%s: %s (status %d)" % (where, pasm_strerror(code), code))
        self.code = code


_lib = None


def header_symbols():
    """Names of the functions include/pasm.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(pasm_\w+)\s*\(", text, re.M)))


def load_library():
    """Load libpasm.so (built by paper_1908_10251_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libpasm.so is not built (%s); run `python -m paper_1908_10251_gb300.build`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    sig = {
        "pasm_default_opts": (None, [ctypes.POINTER(pasm_opts)]),
        "pasm_setup": (I, [ctypes.POINTER(P), I, ctypes.POINTER(pasm_csr), ctypes.POINTER(pasm_csr),
                           ctypes.POINTER(pasm_csr), ctypes.POINTER(pasm_opts), P]),
        "pasm_init": (I, [P, I, ctypes.c_double, P, P]),
        "pasm_step": (I, [P, ctypes.POINTER(I)]),
        "pasm_get": (I, [P, P, P, P, P]),
        "pasm_solve": (I, [P, I, ctypes.c_double, P, P, P, P, P, P]),
        "pasm_bvp": (I, [P, P, P, P]),
        "pasm_augmented": (I, [P, P, P, P, P, P, P]),
        "pasm_coarse_eigs": (I, [P, P, P]),
        "pasm_project": (I, [P, P, P, P, P]),
        "pasm_projection_kind": (I, [P, ctypes.POINTER(I)]),
        "pasm_secular_stats": (I, [P, P]),
        "pasm_residuals": (I, [P, P]),
        "pasm_tiles": (I, [P, I, P]),
        "pasm_tile_rows": (I, [P, I, P]),
        "pasm_set_tiles": (I, [P, I, P, P]),
        "pasm_debug_waits": (I, [P, I, I]),
        "pasm_sizes": (I, [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
        "pasm_last_launches": (I, [P, ctypes.POINTER(I)]),
        "pasm_trace_step": (I, [P, P, P, P, P]),
        "pasm_kernel_class_name": (ctypes.c_char_p, [I]),
        "pasm_trace_launches": (I, [P, I, P, P, P, P, P, ctypes.POINTER(I)]),
        "pasm_nn_setup": (I, [P, P, P]),
        "pasm_nn_get_weights": (I, [P, P]),
        "pasm_nn_apply": (I, [P, I, I, P, P]),
        "pasm_nn_loss_grad": (I, [P, I, I, P, P, P]),
        "pasm_nn_train": (I, [P, I, I, P, I, ctypes.c_float, P]),
        "pasm_nn_capture_residuals": (I, [P, I, P]),
        "pasm_nn_accepted": (I, [P, P]),
        "pasm_nn_errors": (I, [P, ctypes.POINTER(I)]),
        "pasm_border_noalloc": (I, [I, P, P, P, ctypes.c_int64, P, P, P, ctypes.c_int64, I, P, P, P, P, P, P]),
        "pasm_batch_setup": (I, [ctypes.POINTER(P), I, P, P, P, P, ctypes.POINTER(pasm_opts), P]),
        "pasm_batch_solve": (I, [P, P, ctypes.c_double, P, P, P, P, ctypes.POINTER(I)]),
        "pasm_batch_captures": (I, [P, ctypes.POINTER(I)]),
        "pasm_batch_set_max_steps": (I, [P, I]),
        "pasm_batch_destroy": (None, [P]),
        "pasm_destroy": (None, [P]),
        "pasm_strerror": (ctypes.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, dtype=np.float64):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):                       # torch tensor
        want = {np.float64: "torch.float64", np.int32: "torch.int32", np.float32: "torch.float32"}[dtype]
        if str(a.dtype) != want or not a.is_contiguous():
            raise TypeError("tensor must be contiguous %s" % want)
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("array must be a C-contiguous numpy %s array" % np.dtype(dtype))
    return a.ctypes.data


def _check(code: int, where: str, allow=()):
    if code != PASM_OK and code not in allow:
        raise PasmError(code, where)
    return code


class Context:
    """Owns a pasm_ctx* and the host copies handed to pasm_setup."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        try:
            pasm_destroy(self)
        except Exception:
            pass


def _csr(m):
    indptr = np.ascontiguousarray(m.indptr, dtype=np.int32)
    indices = np.ascontiguousarray(m.indices, dtype=np.int32)
    data = np.ascontiguousarray(m.data, dtype=np.float64)
    s = pasm_csr(int(m.shape[0]), int(m.shape[1]), int(data.size), indptr.ctypes.data,
                 indices.ctypes.data if data.size else None, data.ctypes.data if data.size else None)
    return s, (indptr, indices, data)


def pasm_default_opts(**overrides) -> pasm_opts:
    o = pasm_opts()
    load_library().pasm_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def pasm_setup(A, M, P, opts=None, stream=None) -> Context:
    """A, M: per-level CSR matrices (coarsest first), P: interpolations
    P[l]: level l -> l+1; objects with indptr/indices/data/shape (scipy CSR)."""
    lib = load_library()
    L = len(A)
    keep = []
    arrA = (pasm_csr * L)(); arrM = (pasm_csr * L)(); arrP = (pasm_csr * max(L - 1, 1))()
    for l in range(L):
        arrA[l], k1 = _csr(A[l]); arrM[l], k2 = _csr(M[l]); keep += [k1, k2]
    for l in range(L - 1):
        arrP[l], k3 = _csr(P[l]); keep.append(k3)
    h = ctypes.c_void_p()
    o = opts if opts is not None else pasm_default_opts()
    _check(lib.pasm_setup(ctypes.byref(h), L, arrA, arrM, arrP, ctypes.byref(o), stream), "pasm_setup")
    return Context(h, keep)


def pasm_init(ctx: Context, k: int, tol: float, lambda0=None, U0=None):
    _check(load_library().pasm_init(ctx.handle, k, tol, _ptr(lambda0), _ptr(U0)), "pasm_init")


def pasm_step(ctx: Context) -> int:
    n = ctypes.c_int(0)
    _check(load_library().pasm_step(ctx.handle, ctypes.byref(n)), "pasm_step")
    return n.value


def pasm_step_async(ctx: Context):
    """pasm_step without reading the active count back (no synchronisation)."""
    _check(load_library().pasm_step(ctx.handle, None), "pasm_step")


def pasm_get(ctx: Context, lam=None, U=None, steps=None, status=None):
    _check(load_library().pasm_get(ctx.handle, _ptr(lam), _ptr(U), _ptr(steps, np.int32), _ptr(status, np.int32)),
           "pasm_get")


def pasm_solve(ctx: Context, k: int, tol: float, lambda0=None, U0=None, lambda_out=None, U_out=None,
               steps_out=None, status_out=None) -> int:
    return _check(load_library().pasm_solve(ctx.handle, k, tol, _ptr(lambda0), _ptr(U0), _ptr(lambda_out),
                                            _ptr(U_out), _ptr(steps_out, np.int32), _ptr(status_out, np.int32)),
                  "pasm_solve", allow=(PASM_ENOTCONV,))


def pasm_bvp(ctx: Context, lam, U, Uhat):
    _check(load_library().pasm_bvp(ctx.handle, _ptr(lam), _ptr(U), _ptr(Uhat)), "pasm_bvp")


def pasm_augmented(ctx: Context, lam_prev, Uhat, lambda_out=None, U_out=None, beta=None, zeta=None):
    _check(load_library().pasm_augmented(ctx.handle, _ptr(lam_prev), _ptr(Uhat), _ptr(lambda_out), _ptr(U_out),
                                         _ptr(beta), _ptr(zeta)), "pasm_augmented")


def pasm_project(ctx: Context, b, c, bq, cq):
    """bq = Q^T b, cq = Q^T c (N_H x k each, host or device)."""
    _check(load_library().pasm_project(ctx.handle, _ptr(b), _ptr(c), _ptr(bq), _ptr(cq)), "pasm_project")


def pasm_debug_waits(ctx: Context, skip_mma: int, wait_limit: int):
    """Test hook: make the projection's bounded completion wait run out (see include/pasm.h)."""
    _check(load_library().pasm_debug_waits(ctx.handle, skip_mma, wait_limit), "pasm_debug_waits")


def pasm_tiles(ctx: Context, level: int):
    """{kernel kind: 16-byte chunks per thread (0 = default)} on `level`."""
    out = np.zeros(PASM_TILE_N, dtype=np.int32)
    _check(load_library().pasm_tiles(ctx.handle, level, out.ctypes.data), "pasm_tiles")
    return dict(zip(TILE_KINDS, (int(v) for v in out)))


def pasm_tile_rows(ctx: Context, level: int):
    """{kernel kind: row blocks per thread block (0 = not chosen, runs 1)} on `level`."""
    out = np.zeros(PASM_TILE_N, dtype=np.int32)
    _check(load_library().pasm_tile_rows(ctx.handle, level, out.ctypes.data), "pasm_tile_rows")
    return dict(zip(TILE_KINDS, (int(v) for v in out)))


def pasm_set_tiles(ctx: Context, level: int, chunks: dict, rows: dict = None):
    """Set the tile shapes of `level` from {kind: chunks per thread} and
    {kind: row blocks per block} (kinds missing: 0), as pasm_tiles and
    pasm_tile_rows return them."""
    ch = np.array([int(chunks.get(kk, 0)) for kk in TILE_KINDS], dtype=np.int32)
    rw = np.array([int((rows or {}).get(kk, 0)) for kk in TILE_KINDS], dtype=np.int32)
    _check(load_library().pasm_set_tiles(ctx.handle, level, ch.ctypes.data, rw.ctypes.data), "pasm_set_tiles")


def pasm_projection_kind(ctx: Context) -> int:
    kind = ctypes.c_int(-1)
    _check(load_library().pasm_projection_kind(ctx.handle, ctypes.byref(kind)), "pasm_projection_kind")
    return kind.value


def pasm_residuals(ctx: Context):
    """Per pair ||A u - lambda M u||_2 / (|lambda| ||u||_M) of the current state (k floats)."""
    k = pasm_sizes(ctx)[3]
    out = np.zeros(k, dtype=np.float64)
    _check(load_library().pasm_residuals(ctx.handle, out.ctypes.data), "pasm_residuals")
    return out


def pasm_secular_stats(ctx: Context):
    """(roots solved in the first windows, failed certificates, capped root iterations) since pasm_init."""
    out = np.zeros(3, dtype=np.int32)
    _check(load_library().pasm_secular_stats(ctx.handle, out.ctypes.data), "pasm_secular_stats")
    return tuple(int(v) for v in out)


def pasm_sizes(ctx: Context):
    n = ctypes.c_int64(); nh = ctypes.c_int32(); nl = ctypes.c_int32(); k = ctypes.c_int32()
    _check(load_library().pasm_sizes(ctx.handle, ctypes.byref(n), ctypes.byref(nh), ctypes.byref(nl),
                                     ctypes.byref(k)), "pasm_sizes")
    return n.value, nh.value, nl.value, k.value


def pasm_coarse_eigs(ctx: Context):
    _, nh, _, _ = pasm_sizes(ctx)
    lam = np.zeros(nh)
    Q = np.zeros((nh, nh))
    _check(load_library().pasm_coarse_eigs(ctx.handle, lam.ctypes.data, Q.ctypes.data), "pasm_coarse_eigs")
    return lam, Q


def pasm_last_launches(ctx: Context) -> int:
    n = ctypes.c_int(0)
    _check(load_library().pasm_last_launches(ctx.handle, ctypes.byref(n)), "pasm_last_launches")
    return n.value


PASM_KC_N = 20


def pasm_trace_step(ctx: Context):
    """One traced correction step; returns {class name: (ms, bytes, flops, launches)}."""
    lib = load_library()
    ms = np.zeros(PASM_KC_N); by = np.zeros(PASM_KC_N); fl = np.zeros(PASM_KC_N)
    la = np.zeros(PASM_KC_N, dtype=np.int32)
    _check(lib.pasm_trace_step(ctx.handle, ms.ctypes.data, by.ctypes.data, fl.ctypes.data, la.ctypes.data),
           "pasm_trace_step")
    return {pasm_kernel_class_name(q): (float(ms[q]), float(by[q]), float(fl[q]), int(la[q]))
            for q in range(PASM_KC_N) if la[q] > 0}


def pasm_trace_launches(ctx: Context):
    """Launch list of the last pasm_trace_step: list of (class, rows, ms, bytes, flops)."""
    lib = load_library()
    n = ctypes.c_int(0)
    _check(lib.pasm_trace_launches(ctx.handle, 0, None, None, None, None, None, ctypes.byref(n)), "pasm_trace_launches")
    cls = np.zeros(n.value, dtype=np.int32); rows = np.zeros(n.value, dtype=np.int32)
    ms = np.zeros(n.value, dtype=np.float32); by = np.zeros(n.value); fl = np.zeros(n.value)
    _check(lib.pasm_trace_launches(ctx.handle, n.value, cls.ctypes.data, rows.ctypes.data, ms.ctypes.data,
                                   by.ctypes.data, fl.ctypes.data, ctypes.byref(n)), "pasm_trace_launches")
    return [(pasm_kernel_class_name(int(c)), int(r), float(t), float(b), float(f))
            for c, r, t, b, f in zip(cls, rows, ms, by, fl)]


def pasm_kernel_class_name(cls: int) -> str:
    return load_library().pasm_kernel_class_name(cls).decode()


def pasm_nn_setup(ctx: Context, nx, weights):
    """nx: per-level grid width (0 = level not used); weights: 2592 float32."""
    nx = np.ascontiguousarray(nx, dtype=np.int32)
    _check(load_library().pasm_nn_setup(ctx.handle, nx.ctypes.data, _ptr(weights, np.float32)), "pasm_nn_setup")


def pasm_nn_get_weights(ctx: Context):
    w = np.zeros(NN_WEIGHTS, dtype=np.float32)
    _check(load_library().pasm_nn_get_weights(ctx.handle, w.ctypes.data), "pasm_nn_get_weights")
    return w


def pasm_nn_apply(ctx: Context, level: int, R, D):
    _check(load_library().pasm_nn_apply(ctx.handle, level, R.shape[1], _ptr(R, np.float32), _ptr(D, np.float32)),
           "pasm_nn_apply")


def pasm_nn_loss_grad(ctx: Context, level: int, R):
    loss = np.zeros(1)
    grad = np.zeros(NN_WEIGHTS, dtype=np.float32)
    _check(load_library().pasm_nn_loss_grad(ctx.handle, level, R.shape[1], _ptr(R, np.float32), loss.ctypes.data,
                                            grad.ctypes.data), "pasm_nn_loss_grad")
    return float(loss[0]), grad


def pasm_nn_train(ctx: Context, level: int, R, iters: int, lr: float):
    losses = np.zeros(max(iters, 1))
    _check(load_library().pasm_nn_train(ctx.handle, level, R.shape[1], _ptr(R, np.float32), iters, lr,
                                        losses.ctypes.data), "pasm_nn_train")
    return losses[:iters]


def pasm_nn_capture_residuals(ctx: Context, level: int, R_out):
    _check(load_library().pasm_nn_capture_residuals(ctx.handle, level, _ptr(R_out, np.float32)),
           "pasm_nn_capture_residuals")


def pasm_nn_accepted(ctx: Context, k: int):
    out = np.zeros(k, dtype=np.int32)
    _check(load_library().pasm_nn_accepted(ctx.handle, out.ctypes.data), "pasm_nn_accepted")
    return out


def pasm_nn_errors(ctx: Context) -> int:
    n = ctypes.c_int(0)
    _check(load_library().pasm_nn_errors(ctx.handle, ctypes.byref(n)), "pasm_nn_errors")
    return n.value


def pasm_border_noalloc(n, A_row_ptr, A_col, A_val, M_row_ptr, M_col, M_val, k, X, YA, YM, beta, zeta,
                        stream=None):
    """Bordering products with no device allocation (every argument is caller
    device memory, e.g. torch CUDA tensors); see include/pasm.h."""
    _check(load_library().pasm_border_noalloc(
        n, _ptr(A_row_ptr, np.int32), _ptr(A_col, np.int32), _ptr(A_val), A_val.numel() if hasattr(A_val, "numel")
        else A_val.size, _ptr(M_row_ptr, np.int32), _ptr(M_col, np.int32), _ptr(M_val),
        M_val.numel() if hasattr(M_val, "numel") else M_val.size, k, _ptr(X), _ptr(YA), _ptr(YM), _ptr(beta),
        _ptr(zeta), stream), "pasm_border_noalloc")


class Batch:
    """Owns a pasm_batch* and the host CSR copies of every problem."""

    def __init__(self, handle, keep, sizes):
        self.handle = handle
        self._keep = keep
        self.sizes = sizes

    def __del__(self):
        try:
            pasm_batch_destroy(self)
        except Exception:
            pass


def pasm_batch_setup(problems, opts=None, stream=None) -> Batch:
    """problems: list of (A_levels, M_levels, P_levels) (coarsest first)."""
    lib = load_library()
    n = len(problems)
    keep, aptr, mptr, pptr, nlev, sizes = [], [], [], [], [], []
    for A, M, P in problems:
        L = len(A)
        arrA = (pasm_csr * L)(); arrM = (pasm_csr * L)(); arrP = (pasm_csr * max(L - 1, 1))()
        for l in range(L):
            arrA[l], k1 = _csr(A[l]); arrM[l], k2 = _csr(M[l]); keep += [k1, k2]
        for l in range(L - 1):
            arrP[l], k3 = _csr(P[l]); keep.append(k3)
        keep += [arrA, arrM, arrP]
        aptr.append(ctypes.addressof(arrA)); mptr.append(ctypes.addressof(arrM)); pptr.append(ctypes.addressof(arrP))
        nlev.append(L)
        sizes.append(A[-1].shape[0])
    AP = (ctypes.c_void_p * n)(*aptr); MP = (ctypes.c_void_p * n)(*mptr); PP = (ctypes.c_void_p * n)(*pptr)
    NL = (ctypes.c_int * n)(*nlev)
    keep += [AP, MP, PP, NL]
    h = ctypes.c_void_p()
    o = opts if opts is not None else pasm_default_opts()
    _check(lib.pasm_batch_setup(ctypes.byref(h), n, NL, AP, MP, PP, ctypes.byref(o), stream), "pasm_batch_setup")
    return Batch(h, keep, sizes)


def pasm_batch_solve(batch: Batch, ks, tol: float):
    """Returns (code, lams, Us, steps, statuses, rounds) with host numpy outputs per problem."""
    lib = load_library()
    n = len(batch.sizes)
    lams = [np.zeros(k) for k in ks]
    Us = [np.zeros((nf, k)) for nf, k in zip(batch.sizes, ks)]
    steps = [np.zeros(k, dtype=np.int32) for k in ks]
    stats = [np.zeros(k, dtype=np.int32) for k in ks]
    arr = lambda xs: (ctypes.c_void_p * n)(*[x.ctypes.data for x in xs])  # noqa: E731
    K = (ctypes.c_int * n)(*ks)
    rounds = ctypes.c_int(0)
    code = _check(lib.pasm_batch_solve(batch.handle, K, tol, arr(lams), arr(Us), arr(steps), arr(stats),
                                       ctypes.byref(rounds)), "pasm_batch_solve", allow=(PASM_ENOTCONV,))
    return code, lams, Us, steps, stats, rounds.value


def pasm_batch_set_max_steps(batch: Batch, max_steps: int):
    _check(load_library().pasm_batch_set_max_steps(batch.handle, max_steps), "pasm_batch_set_max_steps")


def pasm_batch_captures(batch: Batch) -> int:
    """Step graphs the batch has captured (one per change of the unfinished set)."""
    n = ctypes.c_int(0)
    _check(load_library().pasm_batch_captures(batch.handle, ctypes.byref(n)), "pasm_batch_captures")
    return n.value


def pasm_batch_destroy(batch: Batch):
    if batch.handle is not None and batch.handle.value:
        load_library().pasm_batch_destroy(batch.handle)
    batch.handle = ctypes.c_void_p()


def pasm_destroy(ctx: Context):
    if ctx.handle is not None and ctx.handle.value:
        load_library().pasm_destroy(ctx.handle)
    ctx.handle = ctypes.c_void_p()


def pasm_strerror(code: int) -> str:
    try:
        return load_library().pasm_strerror(code).decode()
    except Exception:
        return "status %d" % code
