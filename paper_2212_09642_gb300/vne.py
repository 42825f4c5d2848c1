"""ctypes binding of the libvne C ABI (include/vne.h).

Argument marshalling only: every step of the computation runs in libvne's
CUDA kernels.  Function names follow the C ABI.  Host arrays are NumPy
arrays; device arrays may be passed as CUDA tensors (their ``data_ptr``) or
integer addresses.  The binding raises :class:`VneError` for every non-zero
status, with the library's message.

The shared library is built in-tree by ``__graft_entry__.build()`` (or
``paper_2212_09642_gb300._build.build()``); importing this module without it
raises immediately -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvne.so")

VNE_OK = 0
VNE_EINVAL = 1
VNE_ENOMEM = 2
VNE_ENOTSYM = 3
VNE_ENOCONVERGE = 4
VNE_ETIMEOUT = 5
VNE_EDEVICE = 6
VNE_EUNSUPPORTED = 7

VNE_FP64 = 0x1
VNE_FP32 = 0x2
VNE_NORMALIZE_TRACE = 0x4
VNE_IS_LAPLACIAN = 0x8
VNE_INPUT_DEVICE = 0x10
VNE_REORDER = 0x20
VNE_REORDER_RCM = 0x80
VNE_CHECK_SYMMETRY = 0x40
VNE_VECTORS_DEVICE = 0x1


class VneError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"libvne status {status}: {message}")
        self.status = status


class vne_options(ctypes.Structure):
    _fields_ = [("reorth", ctypes.c_int32), ("block", ctypes.c_int32), ("panel", ctypes.c_int32),
                ("item_nnz", ctypes.c_int32), ("n_inf_poles", ctypes.c_int32), ("cg_max_iter", ctypes.c_int32),
                ("cg_tol", ctypes.c_double), ("breakdown_tol", ctypes.c_double),
                ("step_variant", ctypes.c_int32), ("interleave", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("probe_offset", ctypes.c_int32), ("check_every", ctypes.c_int32), ("quad_tol", ctypes.c_double),
                ("spectrum_min", ctypes.c_double), ("gaussian_probes", ctypes.c_int32),
                ("items_per_warp", ctypes.c_int32), ("sketch_steps", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_PD = ctypes.POINTER(ctypes.c_double)
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PI64 = ctypes.POINTER(ctypes.c_int64)


_COLORING_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                ctypes.POINTER(ctypes.c_int32))


def _declare(lib):
    st = ctypes.c_int32
    sig = {
        "vne_options_default": (None, [ctypes.POINTER(vne_options)]),
        "vne_version": (ctypes.c_char_p, []),
        "vne_ctx_create": (st, [ctypes.c_int32, ctypes.POINTER(_P)]),
        "vne_ctx_destroy": (st, [_P]),
        "vne_ctx_set_stream": (st, [_P, _P]),
        "vne_last_error": (ctypes.c_char_p, [_P]),
        "vne_create_density_matrix": (st, [_P, ctypes.c_int64, _P, _P, _P, ctypes.c_uint32, ctypes.POINTER(_P)]),
        "vne_matrix_destroy": (st, [_P]),
        "vne_matrix_info": (st, [_P, _PI64, _PI64, _PD, _PD]),
        "vne_quadform_batch": (st, [_P, _P, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32, _P, ctypes.c_int32,
                                    ctypes.POINTER(vne_options), _PD, _PD]),
        "vne_entropy_hutchinson": (st, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.POINTER(vne_options), _PD, _PD, _PD]),
        "vne_entropy_hutchpp": (st, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                     ctypes.POINTER(vne_options), _PD, _PD]),
        "vne_hutchpp_sketch": (st, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                    ctypes.POINTER(vne_options), ctypes.c_uint32, _P]),
        "vne_hutchpp_project": (st, [_P, _P, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(vne_options),
                                     _PD, _PI32, _PI32]),
        "vne_entropy_probing": (st, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32,
                                     ctypes.POINTER(vne_options), _PD, _PI32]),
        "vne_greedy_coloring": (st, [ctypes.c_int64, _P, _P, ctypes.c_int32, _P, _PI32]),
        "vne_matrix_coloring": (st, [_P, ctypes.c_int32, _P, _PI32, _PI32]),
        "vne_gaussian_probes": (st, [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P]),
        "vne_block_gram": (st, [_P, _P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P]),
        "vne_block_apply": (st, [_P, _P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_int64,
                                 ctypes.c_double]),
        "vne_entropy_probing_auto": (st, [_P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _COLORING_FN, _P,
                                          ctypes.POINTER(vne_options), _PD, ctypes.POINTER(vne_probing_report)]),
        "vne_spmm": (st, [_P, _P, _P, ctypes.c_int32]),
        "vne_tridiag_quadrature": (st, [_P, _P, _P, _P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _P]),
        "vne_rademacher": (st, [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]),
        "vne_batch_hutchinson": (st, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.POINTER(vne_options), _P, _P]),
        "vne_ctx_profile": (st, [_P, ctypes.c_int32]),
        "vne_server_create": (st, [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.POINTER(vne_options), ctypes.POINTER(_P)]),
        "vne_server_destroy": (st, [_P]),
        "vne_server_submit": (st, [_P, _P, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32, _PI32]),
        "vne_server_step": (st, [_P, _PI32, _PI32]),
        "vne_server_result": (st, [_P, ctypes.c_int32, _PI32, _PD, _PD, _PI64, _P]),
        "vne_server_info": (st, [_P, _PI32, _PI32, ctypes.POINTER(ctypes.c_uint64)]),
        "vne_quadform_rational": (st, [_P, _P, ctypes.c_int32, ctypes.c_uint32, _P, ctypes.c_int32,
                                       ctypes.POINTER(vne_options), _PD, _P, _P]),
        "vne_autotune": (st, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(vne_options), _PD]),
        "vne_quadform_noalloc": (st, [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
        "vne_ctx_stats": (st, [_P, _PI64, _P]),
        "vne_ctx_graph_stats": (st, [_P, _PI64, _PI64]),
        "vne_ctx_last_steps": (st, [_P, _PI32]),
        "vne_ctx_last_poly_dim": (st, [_P, _PI32]),
        "vne_quadrature_bounds": (st, [_P, _P, _P, _P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int32, _P, _P, _P]),
        "vne_debug_fail_allocation": (st, [ctypes.c_int64]),
        "vne_debug_live_allocations": (st, [_PI64, _PI64]),
        "vne_debug_tensor_wait_limit": (st, [ctypes.c_int64]),
        "vne_measure_gather": (st, [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_int32, _PD]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return sig


def load():
    """Load libvne.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        _declare(lib)
        _lib = lib
    return _lib


def exported_symbols():
    """Names of the C-ABI functions this binding declares."""
    return list(_SIGNATURES)


_SIGNATURES = ["vne_options_default", "vne_version", "vne_ctx_create", "vne_ctx_destroy", "vne_ctx_set_stream",
               "vne_last_error", "vne_create_density_matrix", "vne_matrix_destroy", "vne_matrix_info",
               "vne_quadform_batch", "vne_entropy_hutchinson", "vne_entropy_hutchpp", "vne_hutchpp_sketch",
               "vne_hutchpp_project", "vne_entropy_probing",
               "vne_greedy_coloring", "vne_matrix_coloring", "vne_gaussian_probes", "vne_block_gram", "vne_block_apply", "vne_entropy_probing_auto", "vne_spmm", "vne_tridiag_quadrature", "vne_quadrature_bounds", "vne_rademacher",
               "vne_batch_hutchinson", "vne_ctx_profile", "vne_ctx_stats",
               "vne_ctx_graph_stats", "vne_ctx_last_steps", "vne_ctx_last_poly_dim", "vne_measure_gather", "vne_quadform_noalloc", "vne_autotune", "vne_quadform_rational",
               "vne_server_create", "vne_server_destroy", "vne_server_submit", "vne_server_step",
               "vne_server_result", "vne_server_info", "vne_debug_fail_allocation", "vne_debug_live_allocations",
               "vne_debug_tensor_wait_limit"]


def _check(status, ctx=None):
    if status != VNE_OK:
        msg = load().vne_last_error(ctx).decode() if ctx else ""
        raise VneError(status, msg)


def _ptr(a):
    """Address of a NumPy array, a CUDA tensor, an int address or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def options(**kw) -> vne_options:
    o = vne_options()
    load().vne_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def vne_version() -> str:
    return load().vne_version().decode()


def vne_ctx_create(device: int = 0):
    h = _P()
    _check(load().vne_ctx_create(int(device), ctypes.byref(h)))
    return h


def vne_ctx_destroy(ctx):
    _check(load().vne_ctx_destroy(ctx))


def vne_ctx_set_stream(ctx, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t address, or None."""
    s = getattr(stream, "cuda_stream", stream)
    _check(load().vne_ctx_set_stream(ctx, s), ctx)


def vne_create_density_matrix(ctx, n, row_ptr, col_idx, vals=None, flags=VNE_FP32):
    if not (flags & VNE_INPUT_DEVICE):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        if vals is not None:
            vals = np.ascontiguousarray(vals, dtype=np.float64)
    h = _P()
    _check(load().vne_create_density_matrix(ctx, int(n), _ptr(row_ptr), _ptr(col_idx), _ptr(vals), int(flags),
                                            ctypes.byref(h)), ctx)
    return h


def vne_matrix_destroy(mat):
    _check(load().vne_matrix_destroy(mat))


def vne_matrix_info(mat):
    n, nnz = ctypes.c_int64(), ctypes.c_int64()
    tr, nb = ctypes.c_double(), ctypes.c_double()
    _check(load().vne_matrix_info(mat, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(tr), ctypes.byref(nb)))
    return n.value, nnz.value, tr.value, nb.value


def vne_quadform_batch(ctx, mat, vectors, krylov_steps, opt=None, want_alpha_beta=False, device=False, k=None):
    """psi (and optionally alpha/beta, shape [k, 2m]) for the columns of ``vectors`` ([n, k])."""
    if device:
        kk = int(k if k is not None else vectors.shape[1])
        vp = _ptr(vectors)
        flags = VNE_VECTORS_DEVICE
    else:
        vectors = np.ascontiguousarray(vectors, dtype=np.float64)
        kk = vectors.shape[1]
        vp = _ptr(vectors)
        flags = 0
    psi = np.zeros(kk)
    ab = np.zeros((kk, 2 * krylov_steps)) if want_alpha_beta else None
    o = opt if opt is not None else options()
    _check(load().vne_quadform_batch(mat, vp, kk, flags, int(krylov_steps), None, 0, ctypes.byref(o),
                                     psi.ctypes.data_as(_PD), ab.ctypes.data_as(_PD) if ab is not None else None), ctx)
    return (psi, ab) if want_alpha_beta else psi


def vne_quadform_rational(ctx, mat, vectors, shifts=None, num_shifts=None, opt=None):
    """(psi, cg_iterations [S, k], residuals [S, k]) for the columns of ``vectors`` ([n, k])."""
    vectors = np.ascontiguousarray(vectors, dtype=np.float64)
    k = vectors.shape[1]
    sh = None if shifts is None else np.ascontiguousarray(shifts, dtype=np.float64)
    S = len(sh) if sh is not None else int(num_shifts or 8)
    psi = np.zeros(k)
    its = np.zeros((S, k), dtype=np.int32)
    res = np.zeros((S, k))
    o = opt if opt is not None else options()
    _check(load().vne_quadform_rational(mat, _ptr(vectors), k, 0, _ptr(sh), S, ctypes.byref(o),
                                        psi.ctypes.data_as(_PD), _ptr(its), _ptr(res)), ctx)
    return psi, its, res


def vne_entropy_hutchinson(ctx, mat, num_vectors, krylov_steps, seed, opt=None, want_psi=False):
    est, se = ctypes.c_double(), ctypes.c_double()
    psi = np.zeros(num_vectors) if want_psi else None
    o = opt if opt is not None else options()
    _check(load().vne_entropy_hutchinson(mat, int(num_vectors), int(krylov_steps), int(seed) & (2**64 - 1),
                                         ctypes.byref(o), ctypes.byref(est), ctypes.byref(se),
                                         psi.ctypes.data_as(_PD) if psi is not None else None), ctx)
    return (est.value, se.value, psi) if want_psi else (est.value, se.value)


def vne_entropy_hutchpp(ctx, mat, sketch_cols, hutch_vectors, krylov_steps, seed, opt=None):
    est = ctypes.c_double()
    parts = np.zeros(3)
    o = opt if opt is not None else options()
    _check(load().vne_entropy_hutchpp(mat, int(sketch_cols), int(hutch_vectors), int(krylov_steps),
                                      int(seed) & (2**64 - 1), ctypes.byref(o), ctypes.byref(est),
                                      parts.ctypes.data_as(_PD)), ctx)
    return est.value, parts


def vne_hutchpp_sketch(ctx, mat, col_begin, ncols, krylov_steps, seed, fp64, opt=None, out=None):
    """Columns [col_begin, col_begin + ncols) of the Hutch++ sketch f(A) Omega,
    shape [n, ncols] in the caller's node order (float64 for an FP64 matrix,
    float32 for FP32).  ``out``: a contiguous CUDA tensor of that shape and
    dtype (the sketch stays on the device), else a new NumPy array."""
    n = vne_matrix_info(mat)[0]
    dt = np.float64 if fp64 else np.float32
    o = opt if opt is not None else options()
    if out is not None:
        _require_device_block(out, (n, ncols), dt)
        flags, dst = VNE_VECTORS_DEVICE, out
    else:
        flags, dst = 0, np.zeros((n, ncols), dtype=dt)
    _check(load().vne_hutchpp_sketch(mat, int(col_begin), int(ncols), int(krylov_steps), int(seed) & (2**64 - 1),
                                     ctypes.byref(o), flags, _ptr(dst)), ctx)
    return dst


def vne_hutchpp_project(ctx, mat, Y, sketch_cols, hutch_vectors, krylov_steps, seed, col_begin=0, ncols=None,
                        opt=None):
    """(psi [ncols], pivots [N_r], rank) of the Hutch++ quadratic forms with index
    in [col_begin, col_begin + ncols) of [q_1..q_Nr | g'_1..g'_NH], from the
    whole sketch Y ([n, N_r], a NumPy array or a contiguous CUDA tensor)."""
    total = int(sketch_cols) + int(hutch_vectors)
    ncols = total - int(col_begin) if ncols is None else int(ncols)
    if hasattr(Y, "data_ptr"):
        if not Y.is_cuda or not Y.is_contiguous() or Y.dim() != 2 or Y.shape[1] != sketch_cols:
            raise VneError(VNE_EINVAL, "Y must be a contiguous CUDA tensor of shape [n, N_r]")
        flags = VNE_VECTORS_DEVICE
    else:
        Y = np.ascontiguousarray(Y)
        if Y.ndim != 2 or Y.shape[1] != sketch_cols or Y.dtype not in (np.float32, np.float64):
            raise VneError(VNE_EINVAL, "Y must be a float32/float64 array of shape [n, N_r]")
        flags = 0
    psi = np.zeros(max(ncols, 0))
    piv = np.zeros(int(sketch_cols), dtype=np.int32)
    r = ctypes.c_int32()
    o = opt if opt is not None else options()
    _check(load().vne_hutchpp_project(mat, _ptr(Y), flags, int(sketch_cols), int(hutch_vectors), int(krylov_steps),
                                      int(seed) & (2**64 - 1), int(col_begin), ncols, ctypes.byref(o),
                                      psi.ctypes.data_as(_PD), piv.ctypes.data_as(_PI32), ctypes.byref(r)), ctx)
    return psi, piv, r.value


def _require_device_block(t, shape, dtype):
    """A contiguous CUDA tensor of the given shape and NumPy dtype, else VneError."""
    names = {np.float64: "torch.float64", np.float32: "torch.float32", np.int32: "torch.int32"}
    ok = (hasattr(t, "data_ptr") and t.is_cuda and t.is_contiguous() and tuple(t.shape) == tuple(shape)
          and str(t.dtype) == names[dtype])
    if not ok:
        raise VneError(VNE_EINVAL, f"expected a contiguous CUDA tensor {tuple(shape)} of {names[dtype]}")


def vne_entropy_probing(ctx, mat, coloring=None, distance=1, krylov_steps=30, opt=None, shifts=None,
                        num_shifts=0):
    """Probing estimate; with shifts (or num_shifts > 0 for the default poles) the
    quadratic forms use the rational Krylov space (multi-shift CG)."""
    est = ctypes.c_double()
    s = ctypes.c_int32()
    o = opt if opt is not None else options()
    cp = None
    if coloring is not None:
        coloring = np.ascontiguousarray(coloring, dtype=np.int32)
        cp = _ptr(coloring)
    sh = None if shifts is None else np.ascontiguousarray(shifts, dtype=np.float64)
    S = len(sh) if sh is not None else int(num_shifts)
    _check(load().vne_entropy_probing(mat, cp, int(distance), int(krylov_steps), _ptr(sh), S, ctypes.byref(o),
                                      ctypes.byref(est), ctypes.byref(s)), ctx)
    return est.value, s.value


def vne_greedy_coloring(n, row_ptr, col_idx, distance):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    colors = np.zeros(n, dtype=np.int32)
    s = ctypes.c_int32()
    _check(load().vne_greedy_coloring(int(n), _ptr(row_ptr), _ptr(col_idx), int(distance), _ptr(colors),
                                      ctypes.byref(s)))
    return colors, s.value


class vne_probing_report(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double * 3), ("eps_abs", ctypes.c_double), ("distance", ctypes.c_int32),
                ("num_colors", ctypes.c_int32), ("colors_d", ctypes.c_int32 * 3), ("steps_d", ctypes.c_int32 * 3),
                ("steps_chosen", ctypes.c_int32), ("rule", ctypes.c_int32), ("evaluated", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def vne_entropy_probing_auto(ctx, mat, eps, krylov_steps=60, d_max=64, opt=None, coloring=None):
    """Probing with the heuristic choice of d: (estimate, report dict).
    coloring: optional callable d -> int array of n colours (caller numbering)
    used instead of the device's greedy colouring."""
    est = ctypes.c_double()
    rep = vne_probing_report()
    o = opt if opt is not None else options()
    cb = _COLORING_FN()
    if coloring is not None:
        def _fill(user, d, n, out):
            try:
                c = np.ascontiguousarray(coloring(int(d)), dtype=np.int32)
                if c.shape != (n,) or c.min() < 0:
                    return 0
                ctypes.memmove(out, c.ctypes.data, c.nbytes)
                return int(c.max()) + 1
            except Exception:
                return 0
        cb = _COLORING_FN(_fill)
    _check(load().vne_entropy_probing_auto(mat, float(eps), int(krylov_steps), int(d_max), cb, None,
                                           ctypes.byref(o), ctypes.byref(est), ctypes.byref(rep)), ctx)
    return est.value, dict(T=list(rep.t), eps_abs=rep.eps_abs, d=rep.distance, colors=rep.num_colors,
                           colors_d=list(rep.colors_d), steps_d=list(rep.steps_d), steps=rep.steps_chosen,
                           rule=rep.rule, evaluated=rep.evaluated)


def vne_matrix_coloring(ctx, mat, n, distance):
    """Greedy distance-d colouring of the matrix's graph on the device, in the
    caller's numbering: (colours, s, device rounds; 0 rounds = host sweep)."""
    colors = np.zeros(n, dtype=np.int32)
    s, rounds = ctypes.c_int32(), ctypes.c_int32()
    _check(load().vne_matrix_coloring(mat, int(distance), _ptr(colors), ctypes.byref(s), ctypes.byref(rounds)), ctx)
    return colors, s.value, rounds.value


def vne_block_gram(ctx, X, kx, Y, ky, ks, n):
    """C = X^T Y (float64 [kx, ky]) of two device float32 panel-major blocks."""
    C = np.zeros((kx, ky), dtype=np.float64)
    _check(load().vne_block_gram(ctx, _ptr(X), int(kx), _ptr(Y), int(ky), int(ks), int(n), _ptr(C)), ctx)
    return C


def vne_block_apply(ctx, In, kin, M, kout, In2, Out, ks, n, coef=1.0):
    """Out = In2 + coef In M on device float32 panel-major blocks (M: host float64 [kin, kout])."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    _check(load().vne_block_apply(ctx, _ptr(In), int(kin), _ptr(M), int(kout), _ptr(In2), _ptr(Out), int(ks), int(n),
                                  float(coef)), ctx)


def vne_gaussian_probes(ctx, seed, n, col_begin, k, out):
    """Fill the device tensor out (float64, [n, k]) with the Gaussian probes."""
    _check(load().vne_gaussian_probes(ctx, int(seed) & (2**64 - 1), int(n), int(col_begin), int(k), _ptr(out)), ctx)


def vne_spmm(ctx, mat, X, Y, k):
    _check(load().vne_spmm(mat, _ptr(X), _ptr(Y), int(k)), ctx)


def vne_tridiag_quadrature(ctx, alpha, beta, norm2, scale):
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    norm2 = np.ascontiguousarray(norm2, dtype=np.float64)
    count, m = alpha.shape
    psi = np.zeros(count)
    _check(load().vne_tridiag_quadrature(ctx, _ptr(alpha), _ptr(beta), _ptr(norm2), float(scale), count, m,
                                         _ptr(psi)), ctx)
    return psi


def vne_quadrature_bounds(ctx, alpha, beta, norm2, scale, lam_min, lam_max, grid=4000):
    """(lower, upper, estimate) of Theorem 4.4 for tridiagonals alpha/beta [count, m] (beta[:, m-1] = beta_m)."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    norm2 = np.ascontiguousarray(norm2, dtype=np.float64)
    count, m = alpha.shape
    lo, hi, est = np.zeros(count), np.zeros(count), np.zeros(count)
    _check(load().vne_quadrature_bounds(ctx, _ptr(alpha), _ptr(beta), _ptr(norm2), float(scale), count, m,
                                        float(lam_min), float(lam_max), int(grid), _ptr(lo), _ptr(hi), _ptr(est)), ctx)
    return lo, hi, est


def vne_rademacher(ctx, seed, n, col_begin, k, out_device, fp64):
    _check(load().vne_rademacher(ctx, int(seed) & (2**64 - 1), int(n), int(col_begin), int(k), int(bool(fp64)),
                                 _ptr(out_device)), ctx)


def vne_batch_hutchinson(ctx, mats, num_vectors, krylov_steps, seed, opt=None):
    arr = (_P * len(mats))(*mats)
    est = np.zeros(len(mats))
    se = np.zeros(len(mats))
    o = opt if opt is not None else options()
    _check(load().vne_batch_hutchinson(arr, len(mats), int(num_vectors), int(krylov_steps), int(seed) & (2**64 - 1),
                                       ctypes.byref(o), _ptr(est), _ptr(se)), ctx)
    return est, se


def vne_autotune(ctx, mat, k, steps=8):
    """Pick the fastest schedule for `mat` (kept as its default); returns (options, ms_per_step)."""
    o = vne_options()
    ms = ctypes.c_double()
    _check(load().vne_autotune(mat, int(k), int(steps), ctypes.byref(o), ctypes.byref(ms)), ctx)
    return o, ms.value


def vne_ctx_profile(ctx, enable=True):
    _check(load().vne_ctx_profile(ctx, int(bool(enable))), ctx)


def vne_ctx_stats(ctx):
    """(launches, {kind: (count, ms, algorithmic bytes)}) for kinds step, update, cg_update, cg_direction."""
    n = ctypes.c_int64()
    st = np.zeros(12)
    _check(load().vne_ctx_stats(ctx, ctypes.byref(n), _ptr(st)), ctx)
    names = ["step", "update", "cg_update", "cg_direction"]
    return n.value, {nm: tuple(st[3 * i:3 * i + 3]) for i, nm in enumerate(names)}


def vne_ctx_graph_stats(ctx):
    """(captured, replayed): step loops captured into CUDA graphs / replayed from them."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().vne_ctx_graph_stats(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def vne_ctx_last_steps(ctx):
    """Lanczos steps taken by the last quadrature call (adaptive mode may stop early)."""
    v = ctypes.c_int32()
    _check(load().vne_ctx_last_steps(ctx, ctypes.byref(v)), ctx)
    return v.value

def vne_ctx_last_poly_dim(ctx):
    k = ctypes.c_int32()
    _check(load().vne_ctx_last_poly_dim(ctx, ctypes.byref(k)), ctx)
    return k.value


def vne_debug_fail_allocation(k):
    """Make the k-th allocation from now on fail (VNE_ENOMEM); 0 switches it off."""
    _check(load().vne_debug_fail_allocation(int(k)))


def vne_debug_live_allocations():
    """(device buffers, pinned host buffers) the library currently holds."""
    d, h = ctypes.c_int64(), ctypes.c_int64()
    _check(load().vne_debug_live_allocations(ctypes.byref(d), ctypes.byref(h)))
    return d.value, h.value


def vne_debug_tensor_wait_limit(polls):
    """Poll limit of the tcgen05 kernels' main-loop waits (< 0: the built-in one)."""
    _check(load().vne_debug_tensor_wait_limit(int(polls)))


def vne_measure_gather(ctx, table_bytes, row_bytes, gathers, stream_bytes=0, reps=3):
    """GB/s of random row gathers from a table of table_bytes (plus a concurrent stream)."""
    g = ctypes.c_double()
    _check(load().vne_measure_gather(ctx, int(table_bytes), int(row_bytes), int(gathers), int(stream_bytes),
                                     int(reps), ctypes.byref(g)), ctx)
    return g.value


def vne_quadform_noalloc(stream, n, row_ptr_dev, col_idx_dev, vectors_dev, k, krylov_steps, psi_dev):
    """Allocation-free FP64 Lanczos quadrature; every array is caller-owned device memory
    (see include/vne.h): row_ptr int32 [n + 1], col_idx int32 [nnz], vectors float64
    [n, k] contiguous, psi float64 [k].  Returns without synchronising the stream."""
    if not (hasattr(row_ptr_dev, "data_ptr") and row_ptr_dev.is_cuda and row_ptr_dev.is_contiguous()
            and str(row_ptr_dev.dtype) == "torch.int32" and row_ptr_dev.numel() == int(n) + 1):
        raise VneError(VNE_EINVAL, "row_ptr must be a contiguous CUDA int32 tensor of n + 1 entries")
    if not (hasattr(col_idx_dev, "data_ptr") and col_idx_dev.is_cuda and col_idx_dev.is_contiguous()
            and str(col_idx_dev.dtype) == "torch.int32"):
        raise VneError(VNE_EINVAL, "col_idx must be a contiguous CUDA int32 tensor")
    _require_device_block(vectors_dev, (int(n), int(k)), np.float64)
    _require_device_block(psi_dev, (int(k),), np.float64)
    s = getattr(stream, "cuda_stream", stream)
    st = load().vne_quadform_noalloc(s, int(n), _ptr(row_ptr_dev), _ptr(col_idx_dev), _ptr(vectors_dev), int(k),
                                     int(krylov_steps), _ptr(psi_dev))
    if st != VNE_OK:
        raise VneError(st, "vne_quadform_noalloc rejected the call (sizes beyond the fixed scratch, or bad arguments)")


def vne_server_create(ctx, hbm_budget_bytes, max_active=64, krylov_steps=40, block_vectors=64, opt=None):
    h = _P()
    o = opt if opt is not None else options()
    _check(load().vne_server_create(ctx, int(hbm_budget_bytes), int(max_active), int(krylov_steps),
                                    int(block_vectors), ctypes.byref(o), ctypes.byref(h)), ctx)
    return h


def vne_server_destroy(srv):
    _check(load().vne_server_destroy(srv))


def vne_server_submit(ctx, srv, mat, rel_eps, seed, max_vectors=8192):
    t = ctypes.c_int32()
    _check(load().vne_server_submit(srv, mat, float(rel_eps), int(seed) & (2**64 - 1), int(max_vectors),
                                    ctypes.byref(t)), ctx)
    return t.value


def vne_server_step(ctx, srv):
    done, act = ctypes.c_int32(), ctypes.c_int32()
    _check(load().vne_server_step(srv, ctypes.byref(done), ctypes.byref(act)), ctx)
    return done.value, act.value


def vne_server_result(srv, ticket):
    """dict(state, estimate, std_error, vectors, submit_tick, admit_tick, done_tick)."""
    state = ctypes.c_int32()
    est, se = ctypes.c_double(), ctypes.c_double()
    nv = ctypes.c_int64()
    ticks = np.zeros(3, dtype=np.int64)
    _check(load().vne_server_result(srv, int(ticket), ctypes.byref(state), ctypes.byref(est), ctypes.byref(se),
                                    ctypes.byref(nv), _ptr(ticks)))
    return dict(state=state.value, estimate=est.value, std_error=se.value, vectors=nv.value,
                submit_tick=int(ticks[0]), admit_tick=int(ticks[1]), done_tick=int(ticks[2]))


def vne_server_info(srv):
    q, a = ctypes.c_int32(), ctypes.c_int32()
    u = ctypes.c_uint64()
    _check(load().vne_server_info(srv, ctypes.byref(q), ctypes.byref(a), ctypes.byref(u)))
    return q.value, a.value, u.value


# ---------------------------------------------------------------------------
# small convenience layer (still marshalling only)

def matrix_from_graph(ctx, graph, fp64=False, reorder=False, extra_flags=0):
    """Density matrix rho = L / tr(L) of a graph pattern (implicit Laplacian).
    reorder: False, True (degree order) or "rcm" (reverse Cuthill-McKee)."""
    ro = VNE_REORDER_RCM if reorder == "rcm" else (VNE_REORDER if reorder else 0)
    flags = (VNE_FP64 if fp64 else VNE_FP32) | ro | extra_flags
    return vne_create_density_matrix(ctx, graph.n, graph.rowptr, graph.col, None, flags)
