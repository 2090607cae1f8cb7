"""Python binding of libsced (include/sced.h): argument marshalling only.

Every step of the symmetry-adapted product runs in the CUDA library; this module
turns numpy arrays and torch CUDA tensors into the plain pointers and sizes of the
C ABI.  There is no fallback: if ``libsced.so`` is missing or cannot be loaded the
import of :func:`lib` raises.

The names follow the C ABI: :func:`build_basis`, :meth:`Basis.apply_H`,
:meth:`Basis.lanczos`, :meth:`Basis.find_rep`.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["lib", "build", "build_basis", "build_basis_from", "Basis", "Batch", "EdError",
           "F64", "F32", "C128", "C64", "LIB_PATH", "SYMBOLS", "build_sectors", "dot_noalloc",
           "axpy_norm", "scale"]

F64, F32, C128, C64 = 0, 1, 2, 3
REORTH = {"local": 0, "none": 1, "full": 2}
LIB_PATH = _build.LIB
# every function declared in include/sced.h
SYMBOLS = ["ed_build_basis", "ed_free_basis", "ed_basis_info", "ed_basis_export",
           "ed_find_rep", "ed_apply_H", "ed_apply_H_rows", "ed_apply_H_host", "ed_lanczos",
           "ed_dot", "ed_count_terms", "ed_expect_classes", "ed_dot_noalloc", "ed_batch_create",
           "ed_batch_set_vectors", "ed_batch_apply", "ed_batch_info", "ed_batch_free",
           "ed_axpy_norm", "ed_scale", "ed_last_error", "ed_version"]

_ERR = {1: "ED_ERR_INVALID", 2: "ED_ERR_UNSTABLE", 3: "ED_ERR_OOM", 4: "ED_ERR_CUDA",
        5: "ED_ERR_TIMEOUT", 6: "ED_ERR_EMPTY", 7: "ED_ERR_UNSUPPORTED"}


class EdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR.get(code, code)}: {msg}")
        self.code = code


class _Lattice(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int32), ("n_sublat", ctypes.c_int32),
                ("n_bonds", ctypes.c_int32), ("n_classes", ctypes.c_int32),
                ("bonds", ctypes.c_void_p), ("bond_class", ctypes.c_void_p)]


class _Group(ctypes.Structure):
    _fields_ = [("n_sym", ctypes.c_int32), ("perm", ctypes.c_void_p), ("flip", ctypes.c_void_p)]


class _Irrep(ctypes.Structure):
    _fields_ = [("phase_denom", ctypes.c_int32), ("phase_num", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("bucket_target", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("share_tables", ctypes.c_void_p), ("reserved", ctypes.c_int64 * 2)]


class _Info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int64), ("is_real", ctypes.c_int32),
                ("n_sites", ctypes.c_int32), ("n_sublat", ctypes.c_int32),
                ("n_sym", ctypes.c_int32), ("n_up", ctypes.c_int32),
                ("n_bonds", ctypes.c_int32), ("n_classes", ctypes.c_int32),
                ("prefix_rank_bits", ctypes.c_int32), ("prefix_raw_bits", ctypes.c_int32),
                ("postfix_bits", ctypes.c_int32), ("n_keys", ctypes.c_int64),
                ("max_bucket", ctypes.c_int64), ("table_bytes", ctypes.c_int64),
                ("index_bytes", ctypes.c_int64), ("basis_bytes", ctypes.c_int64),
                ("sym_list_len", ctypes.c_int64), ("build_ms", ctypes.c_double)]


class _LOpts(ctypes.Structure):
    _fields_ = [("max_steps", ctypes.c_int32), ("fixed_steps", ctypes.c_int32),
                ("tol", ctypes.c_double), ("dtype", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("v0", ctypes.c_void_p), ("psi", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p), ("beta", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("work", ctypes.c_void_p),
                ("work_bytes", ctypes.c_int64), ("tol_residual", ctypes.c_double),
                ("reorth", ctypes.c_int32), ("reserved1", ctypes.c_int32),
                ("krylov", ctypes.c_void_p), ("krylov_bytes", ctypes.c_int64)]


class _LRes(ctypes.Structure):
    _fields_ = [("E0", ctypes.c_double), ("steps", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("rq", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_apply", ctypes.c_double),
                ("ms_reorth", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libsced.so for sm_103a in-tree."""
    return _build.build(force=force, verbose=verbose)


def lib():
    """Load libsced.so (raises when it is missing: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libsced.so not built ({LIB_PATH}); run "
                                  "python -c 'import __graft_entry__ as g; g.build()'")
            L = ctypes.CDLL(LIB_PATH)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            L.ed_build_basis.argtypes = [vp, vp, vp, i32, vp, vp, ctypes.POINTER(vp)]
            L.ed_free_basis.argtypes = [vp]
            L.ed_free_basis.restype = None
            L.ed_basis_info.argtypes = [vp, vp]
            L.ed_basis_export.argtypes = [vp, vp, vp]
            L.ed_find_rep.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp, vp, vp]
            L.ed_apply_H.argtypes = [vp, vp, vp, vp, vp, i32, vp]
            L.ed_apply_H_rows.argtypes = [vp, vp, vp, vp, vp, i32, i64, i64, vp]
            L.ed_apply_H_host.argtypes = [vp, vp, vp, vp, vp, i32, vp]
            L.ed_lanczos.argtypes = [vp, vp, vp, vp, vp]
            L.ed_dot.argtypes = [vp, vp, vp, i32, vp, vp]
            L.ed_count_terms.argtypes = [vp, vp, vp, vp]
            L.ed_dot_noalloc.argtypes = [vp, vp, i64, i32, vp, vp]
            L.ed_expect_classes.argtypes = [vp, vp, vp, i32, vp, vp]
            L.ed_batch_create.argtypes = [vp, i32, vp, vp, i32, ctypes.POINTER(vp)]
            L.ed_batch_set_vectors.argtypes = [vp, vp, vp]
            L.ed_batch_apply.argtypes = [vp, vp]
            L.ed_batch_info.argtypes = [vp, vp, vp]
            L.ed_batch_free.argtypes = [vp]
            L.ed_batch_free.restype = None
            L.ed_axpy_norm.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, i64, i32, vp,
                                       i64, vp, vp]
            L.ed_scale.argtypes = [vp, ctypes.c_double, i64, i32, vp]
            L.ed_last_error.restype = ctypes.c_char_p
            L.ed_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise EdError(rc, lib().ed_last_error().decode())


def _dtype_code(t) -> int:
    import torch
    m = {torch.float64: F64, torch.float32: F32, torch.complex128: C128, torch.complex64: C64}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def _np_dtype_code(a) -> int:
    m = {np.dtype(np.float64): F64, np.dtype(np.float32): F32,
         np.dtype(np.complex128): C128, np.dtype(np.complex64): C64}
    if a.dtype not in m:
        raise TypeError(f"unsupported dtype {a.dtype}")
    return m[a.dtype]


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _need(*checks):
    """Refuse, before any pointer is formed, every tensor whose element count is not the
    expected one: checks are (tensor or None, expected count, name)."""
    for t, n, what in checks:
        if t is not None and t.numel() != n:
            raise ValueError(f"{what} has {t.numel()} elements, expected {n}")


def _dev(t, dtype=None, n=None, what="tensor", device=None):
    """Device pointer of a contiguous CUDA tensor, after checking (in this order, so that
    a wrong size is refused before anything else is looked at) its element count ``n``,
    that it lives on CUDA device ``device`` (default: the current one), its layout and
    its dtype.  Nothing reaches the library unless every check passes: a short vector
    would let a kernel read or write past its end."""
    if n is not None and t.numel() != n:
        raise ValueError(f"{what} has {t.numel()} elements, expected {n}")
    if not t.is_cuda:
        raise ValueError(f"{what}: expected a CUDA tensor")
    if device is None:
        import torch
        device = torch.cuda.current_device()
    if t.device.index != device:
        raise ValueError(f"{what} is on cuda:{t.device.index}, expected cuda:{device}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what}: expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


class Basis:
    """A symmetry sector's basis and lookup tables on the current CUDA device."""

    def __init__(self, handle, J, Jz, n_classes, device=None):
        self._h = handle
        self.J = tuple(float(v) for v in J) if J is not None else None
        self.Jz = tuple(float(v) for v in Jz) if Jz is not None else None
        self.n_classes = n_classes
        self.device = device      # CUDA device the basis was built on
        self._info = None

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.ed_free_basis(h)

    def close(self):
        if self._h:
            lib().ed_free_basis(self._h)
            self._h = None

    def info(self) -> dict:
        if self._info is None:
            inf = _Info()
            _check(lib().ed_basis_info(self._h, ctypes.byref(inf)))
            self._info = {k: getattr(inf, k) for k, _ in _Info._fields_}
        return dict(self._info)

    @property
    def dim(self) -> int:
        return int(self.info()["dim"])

    @property
    def is_real(self) -> bool:
        return bool(self.info()["is_real"])

    def export(self):
        """(states uint64[D], stab uint16[D]) as numpy arrays."""
        D = self.dim
        s = np.empty(D, np.uint64)
        t = np.empty(D, np.uint16)
        if D:
            _check(lib().ed_basis_export(self._h, s.ctypes.data, t.ctypes.data))
        return s, t

    def _couplings(self, J, Jz):
        J = self.J if J is None else tuple(float(v) for v in J)
        Jz = (self.Jz if self.Jz is not None else (1.0,) * len(J)) if Jz is None else tuple(float(v) for v in Jz)
        if J is None or len(J) != self.n_classes or len(Jz) != self.n_classes:
            raise ValueError(f"need {self.n_classes} couplings per class")
        return (ctypes.c_double * len(J))(*J), (ctypes.c_double * len(Jz))(*Jz)

    def find_rep(self, states, method=0, stream=None):
        """Representative search on a uint64 CUDA tensor of configurations.

        method 0: Alg. 2 as printed; method 1: the two-level search of the product.
        Returns (rep, sym, phase, stab, index) CUDA tensors.
        """
        import torch
        n = states.numel()
        dev = states.device
        rep = torch.empty(n, dtype=torch.uint64, device=dev)
        sym = torch.empty(n, dtype=torch.int32, device=dev)
        ph = torch.empty(n, dtype=torch.int32, device=dev)
        stab = torch.empty(n, dtype=torch.int32, device=dev)
        idx = torch.empty(n, dtype=torch.int64, device=dev)
        d = self.device
        _check(lib().ed_find_rep(self._h, _dev(states, torch.uint64, device=d, what="states"), n,
                                 int(method), _dev(rep, device=d), _dev(sym, device=d),
                                 _dev(ph, device=d), _dev(stab, device=d), _dev(idx, device=d),
                                 _stream(stream)))
        return rep, sym, ph, stab, idx

    def apply_H(self, x, y=None, J=None, Jz=None, stream=None):
        """y = H x for CUDA tensors (float64/float32/complex128/complex64)."""
        import torch
        D, d = self.dim, self.device
        _need((x, D, "x"), (y, D, "y"))
        px = _dev(x, n=D, what="x", device=d)
        if y is None:
            y = torch.empty_like(x)
        py = _dev(y, x.dtype, n=D, what="y", device=d)
        cJ, cJz = self._couplings(J, Jz)
        _check(lib().ed_apply_H(self._h, cJ, cJz, px, py, _dtype_code(x), _stream(stream)))
        return y

    def apply_H_rows(self, x, row_begin, row_end, y=None, J=None, Jz=None, stream=None):
        import torch
        D, d = self.dim, self.device
        if not 0 <= row_begin <= row_end <= D:
            raise ValueError(f"rows [{row_begin}, {row_end}) outside [0, {D})")
        _need((x, D, "x"), (y, row_end - row_begin, "y"))
        px = _dev(x, n=D, what="x", device=d)
        if y is None:
            y = torch.empty(row_end - row_begin, dtype=x.dtype, device=x.device)
        py = _dev(y, x.dtype, n=row_end - row_begin, what="y", device=d)
        cJ, cJz = self._couplings(J, Jz)
        _check(lib().ed_apply_H_rows(self._h, cJ, cJz, px, py, _dtype_code(x),
                                     int(row_begin), int(row_end), _stream(stream)))
        return y

    def apply_H_host(self, x, y=None, J=None, Jz=None, stream=None):
        """y = H x for HOST numpy arrays (or pinned CPU tensors); copies inside the call."""
        D = self.dim
        if hasattr(x, "data_ptr"):
            import torch
            if y is None:
                y = torch.empty_like(x)
            for t, nm in ((x, "x"), (y, "y")):
                if t.numel() != D or t.is_cuda or not t.is_contiguous():
                    raise ValueError(f"{nm}: expected a contiguous host tensor of {D} elements")
            if y.dtype != x.dtype:
                raise TypeError("x and y differ in dtype")
            code = _dtype_code(x)
            px, py = ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())
        else:
            x = np.ascontiguousarray(x)
            if y is None:
                y = np.empty_like(x)
            if x.size != D or y.size != D or y.dtype != x.dtype or not y.flags.c_contiguous:
                raise ValueError(f"x and y must be contiguous arrays of {D} elements of one dtype")
            code = _np_dtype_code(x)
            px, py = ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(y.ctypes.data)
        cJ, cJz = self._couplings(J, Jz)
        _check(lib().ed_apply_H_host(self._h, cJ, cJz, px, py, code, _stream(stream)))
        return y

    def count_terms(self, stream=None):
        """(exchange terms generated, those with a surviving target) of one product."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ed_count_terms(self._h, ctypes.byref(a), ctypes.byref(b), _stream(stream)))
        return a.value, b.value

    def expect_classes(self, x, Jz=None, stream=None):
        """Re <x|H_c|x> per coupling class c (unit exchange J_c = 1): numpy array."""
        px = _dev(x, n=self.dim, what="x", device=self.device)
        _, cJz = self._couplings((1.0,) * self.n_classes, Jz)
        out = (ctypes.c_double * self.n_classes)()
        _check(lib().ed_expect_classes(self._h, cJz, px, _dtype_code(x), out, _stream(stream)))
        return np.array(out[:])

    def dot(self, x, y, stream=None) -> complex:
        D, d = self.dim, self.device
        _need((x, D, "x"), (y, D, "y"))
        px, py = _dev(x, n=D, what="x", device=d), _dev(y, x.dtype, n=D, what="y", device=d)
        out = (ctypes.c_double * 2)()
        _check(lib().ed_dot(self._h, px, py, _dtype_code(x), out, _stream(stream)))
        return complex(out[0], out[1]) if x.is_complex() else out[0]

    def lanczos(self, J=None, Jz=None, dtype=None, max_steps=300, fixed_steps=0, tol=1e-13,
                seed=1805, v0=None, psi=None, work=None, tol_residual=0.0, reorth="local",
                krylov=None, stream=None):
        """Lanczos ground-state energy; returns a dict (E0, steps, converged, alpha, beta, ...).

        reorth: "local" (default: a second Gram-Schmidt sweep against the last two
        vectors), "none" (three-term recurrence only) or "full" (two sweeps against every
        stored vector; ``krylov`` is a CUDA tensor of (steps + 1) * dim elements of dtype,
        allocated here when None)."""
        import torch
        if dtype is None:
            dtype = torch.float64 if self.is_real else torch.complex128
        code = {torch.float64: F64, torch.float32: F32, torch.complex128: C128,
                torch.complex64: C64}[dtype]
        if reorth not in REORTH:
            raise ValueError(f"reorth must be one of {sorted(REORTH)}")
        m = fixed_steps if fixed_steps > 0 else max_steps
        if reorth == "full" and krylov is None:
            krylov = torch.empty((m + 1) * self.dim, dtype=dtype, device=f"cuda:{self.device}")
        alpha = np.zeros(m)
        beta = np.zeros(m)
        o = _LOpts()
        o.max_steps, o.fixed_steps, o.tol, o.dtype, o.seed = int(max_steps), int(fixed_steps), float(tol), code, int(seed)
        o.tol_residual = float(tol_residual)
        D, d = self.dim, self.device
        _need((v0, D, "v0"), (psi, D, "psi"))
        o.v0 = _dev(v0, dtype, n=D, what="v0", device=d).value if v0 is not None else None
        o.psi = _dev(psi, dtype, n=D, what="psi", device=d).value if psi is not None else None
        o.alpha, o.beta = alpha.ctypes.data, beta.ctypes.data
        o.stream = _stream(stream).value
        if work is not None:
            o.work = _dev(work, device=d, what="work").value
            o.work_bytes = work.numel() * work.element_size()
        o.reorth = REORTH[reorth]
        if krylov is not None:
            o.krylov = _dev(krylov, dtype, device=d, what="krylov").value
            o.krylov_bytes = krylov.numel() * krylov.element_size()
        r = _LRes()
        cJ, cJz = self._couplings(J, Jz)
        _check(lib().ed_lanczos(self._h, cJ, cJz, ctypes.byref(o), ctypes.byref(r)))
        k = r.steps
        return {"E0": r.E0, "steps": k, "converged": bool(r.converged), "rq": r.rq,
                "alpha": alpha[:k].copy(), "beta": beta[:max(k - 1, 0)].copy(),
                "ms_total": r.ms_total, "ms_apply": r.ms_apply, "ms_reorth": r.ms_reorth}


class Batch:
    """Many sectors of one lattice in one persistent launch, each with k vectors
    (ed_batch_*).  Vectors are CUDA float32 (real sectors) or complex64 tensors holding
    dim * k values row-major ([dim][k])."""

    def __init__(self, bases, k=1, J=None, Jz=None):
        self.bases = list(bases)          # the batch refers to them: keep them alive
        b0 = self.bases[0]
        cJ, cJz = b0._couplings(J, Jz)
        arr = (ctypes.c_void_p * len(self.bases))(*[b._h for b in self.bases])
        h = ctypes.c_void_p()
        _check(lib().ed_batch_create(arr, len(self.bases), cJ, cJz, int(k), ctypes.byref(h)))
        self._h, self.k = h, int(k)

    def set_vectors(self, xs, ys):
        import torch
        if len(xs) != len(self.bases) or len(ys) != len(self.bases):
            raise ValueError(f"need one x and one y per sector ({len(self.bases)})")
        for s, (B, x, y) in enumerate(zip(self.bases, xs, ys)):
            _need((x, B.dim * self.k, f"x[{s}]"), (y, B.dim * self.k, f"y[{s}]"))
        for s, (B, x, y) in enumerate(zip(self.bases, xs, ys)):
            n = B.dim * self.k
            dt = torch.float32 if B.is_real else torch.complex64
            if n:
                _dev(x, dt, n=n, what=f"x[{s}]", device=B.device)
                _dev(y, dt, n=n, what=f"y[{s}]", device=B.device)
        px = (ctypes.c_void_p * len(xs))(*[t.data_ptr() if t.numel() else None for t in xs])
        py = (ctypes.c_void_p * len(ys))(*[t.data_ptr() if t.numel() else None for t in ys])
        _check(lib().ed_batch_set_vectors(self._h, px, py))
        self._keep = (xs, ys)

    def apply(self, stream=None):
        _check(lib().ed_batch_apply(self._h, _stream(stream)))

    def info(self):
        r, n = ctypes.c_int32(), ctypes.c_int64()
        _check(lib().ed_batch_info(self._h, ctypes.byref(r), ctypes.byref(n)))
        return {"rows_per_item": r.value, "n_items": n.value}

    def close(self):
        if self._h:
            lib().ed_batch_free(self._h)
            self._h = None

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.ed_batch_free(h)


def dot_noalloc(x, y, out, stream=None):
    """ed_dot_noalloc: <x, y> into the caller's CUDA float64 tensor ``out`` (2 entries:
    re, im) without allocating anything -- for callers that cannot allocate device memory
    at that point (a loop that must not stall the device, or a framework that owns all
    device memory).  Asynchronous; calls that overlap on the device race on the library's
    fixed scratch array."""
    import torch
    if out.dtype != torch.float64 or out.numel() < 2:
        raise TypeError("out must be a CUDA float64 tensor of 2 entries")
    n = x.numel()
    _need((y, n, "y"))
    py = _dev(y, x.dtype, n=n, what="y", device=x.device.index)
    _check(lib().ed_dot_noalloc(_dev(x, what="x"), py, n, _dtype_code(x),
                                _dev(out, what="out", device=x.device.index), _stream(stream)))
    return out


def axpy_norm(w, v, vprev, a, b, scratch, norm2, stream=None):
    """ed_axpy_norm: w <- w - a v - b vprev in place (vprev may be None), ||w||^2 into the
    CUDA float64 tensor ``norm2`` (1 entry), block partials in the CUDA float64 tensor
    ``scratch``.  Asynchronous."""
    import torch
    n = w.numel()
    _need((v, n, "v"), (vprev, n, "vprev"))
    if scratch.dtype != torch.float64 or norm2.dtype != torch.float64 or norm2.numel() < 1:
        raise TypeError("scratch and norm2 must be CUDA float64 tensors")
    d = w.device.index
    pw = _dev(w, what="w", device=d)
    pv = _dev(v, w.dtype, what="v", device=d)
    pp = _dev(vprev, w.dtype, what="vprev", device=d) if vprev is not None else None
    _check(lib().ed_axpy_norm(pw, pv, pp, float(a), float(b), n, _dtype_code(w),
                              _dev(scratch, what="scratch", device=d), scratch.numel(),
                              _dev(norm2, what="norm2", device=d), _stream(stream)))
    return norm2


def scale(x, s, stream=None):
    """ed_scale: x <- s x in place for a CUDA tensor.  Asynchronous."""
    _check(lib().ed_scale(_dev(x, what="x"), float(s), x.numel(), _dtype_code(x), _stream(stream)))
    return x


def build_basis(n_sites, n_sublat, bonds, bond_class, n_classes, perm, phase_num, phase_denom,
                n_up, J=None, Jz=None, bucket_target=None, share_tables=None, flip=None,
                stream=None) -> Basis:
    """Validate a sector, build the sublattice tables and the basis on the current device."""
    bonds = np.ascontiguousarray(bonds, dtype=np.int32)
    bcls = np.ascontiguousarray(bond_class, dtype=np.int32)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    pnum = np.ascontiguousarray(phase_num, dtype=np.int32)
    L = _Lattice(int(n_sites), int(n_sublat), int(bonds.shape[0]), int(n_classes),
                 bonds.ctypes.data, bcls.ctypes.data)
    flip_a = None if flip is None else np.ascontiguousarray(flip, dtype=np.uint8)
    G = _Group(int(perm.shape[0]), perm.ctypes.data, None if flip_a is None else flip_a.ctypes.data)
    R = _Irrep(int(phase_denom), pnum.ctypes.data)
    opts = _Opts()
    opts.bucket_target = int(bucket_target or 0)
    opts.share_tables = share_tables._h if share_tables is not None else None
    h = ctypes.c_void_p()
    _check(lib().ed_build_basis(ctypes.byref(L), ctypes.byref(G), ctypes.byref(R), int(n_up),
                                ctypes.byref(opts), _stream(stream), ctypes.byref(h)))
    import torch
    return Basis(h, J, Jz, int(n_classes), device=torch.cuda.current_device())


def build_basis_from(problem, **kw) -> Basis:
    """build_basis from an object with the fields of a problem descriptor."""
    p = problem
    return build_basis(p.n_sites, p.n_sublat, p.bonds, p.bond_class, p.n_classes, p.perm,
                       p.phase_num, p.phase_denom, p.n_up, J=p.J, Jz=p.Jz,
                       flip=getattr(p, "flip", None), **kw)


def build_sectors(problems, **kw):
    """build_basis_from for many sectors, sharing the one-sublattice table between sectors
    whose lattice and group coincide (the table depends on the group only)."""
    out, first_of_group = [], {}
    for p in problems:
        fl = getattr(p, "flip", None)
        key = (p.n_sites, p.n_sublat, np.asarray(p.perm).tobytes(),
               None if fl is None else np.asarray(fl).tobytes())
        share = first_of_group.get(key) if p.n_sublat == 1 else None
        B = build_basis_from(p, share_tables=share, **kw)
        if p.n_sublat == 1 and key not in first_of_group:
            first_of_group[key] = B
        out.append(B)
    return out
