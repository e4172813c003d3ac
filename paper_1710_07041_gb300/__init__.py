"""GB300-native Wilson-clover SAP-FGMRES (the fine-grid hot path of DD-alpha-AMG).

Thin Python binding over the C ABI in ``include/dd.h``: argument marshalling
only, every computation runs in the CUDA library ``_build/libdd.so``. PyTorch
provides device memory (tensors passed by data pointer) and streams. There is
no CPU fallback: if the library cannot be built or loaded, every call raises.

Names follow the C ABI: ``create_lattice``, ``create_gauge``, ``create_op``,
``apply_D``, ``sap_smooth``, ``solve``, ``pack``/``unpack``, ``server_*``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

F64, F32, F16, BF16 = 0, 1, 2, 3
F64_DF = 4   # apply_D only: FP64 fields in and out, double-float arithmetic
F16N = 5     # FP16 operator tiles, spinors as 16-bit fixed point with a per-site scale
PREC = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16, "f16n": F16N}
HOST, DEVICE = 0, 1
QUEUED, RUNNING, DONE, FAILED, CANCELLED = 0, 1, 2, 3, 4
ERRORS = {0: "DD_OK", -1: "DD_EINVAL", -2: "DD_ENOMEM", -3: "DD_ECUDA", -4: "DD_ENOTCONV",
          -5: "DD_ETIMEOUT", -6: "DD_ECANCELLED", -7: "DD_EBUSY", -8: "DD_ENOTFOUND"}

_lib = None


class DDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SapParams(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("mr_steps", ctypes.c_int), ("x_is_zero", ctypes.c_int),
                ("rhs_tile", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("sap", SapParams), ("inner_reduction", ctypes.c_double), ("where", ctypes.c_int),
                ("use_x0", ctypes.c_int), ("mg", ctypes.c_void_p), ("outer_f64", ctypes.c_int)]


class MgParams(ctypes.Structure):
    _fields_ = [("n_vectors", ctypes.c_int), ("setup_iters", ctypes.c_int), ("coarse_max_iter", ctypes.c_int),
                ("coarse_tol", ctypes.c_double), ("smoother", SapParams)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("cycles", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double), ("est_rel_residual", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_sap", ctypes.c_double), ("ms_dirac", ctypes.c_double),
                ("ms_orth", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("max_batch_rhs", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_void_p), ("b_host", ctypes.c_void_p), ("nrhs", ctypes.c_int),
                ("params", SolveParams)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("rhs_per_s", ctypes.c_double), ("bytes_in_use", ctypes.c_size_t)]


EXPORTS = {
    "dd_version": ([], ctypes.c_char_p),
    "dd_last_error": ([], ctypes.c_char_p),
    "dd_kernel_launches": ([], ctypes.c_uint64),
    "dd_device_status": ([], ctypes.c_int),
    "dd_selftest_wait": ([ctypes.c_int], ctypes.c_int),
    "dd_bench_link_product": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "dd_release_workspace": ([], ctypes.c_int),
    "dd_create_lattice": ([ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                           ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "dd_lattice_volume": ([ctypes.c_void_p], ctypes.c_long),
    "dd_field_bytes": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_size_t),
    "dd_create_gauge": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "dd_create_op": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                      ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "dd_create_op_clover": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)],
                            ctypes.c_int),
    "dd_op_get_clover": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dd_destroy": ([ctypes.c_void_p], None),
    "dd_pack": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                 ctypes.c_void_p], ctypes.c_int),
    "dd_unpack": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                   ctypes.c_void_p], ctypes.c_int),
    "dd_apply_D": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                    ctypes.c_void_p], ctypes.c_int),
    "dd_sap_smooth": ([ctypes.c_void_p, ctypes.POINTER(SapParams), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                       ctypes.c_void_p], ctypes.c_int),
    "dd_sap_smooth_multi": ([ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(SapParams), ctypes.POINTER(ctypes.c_void_p),
                             ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p], ctypes.c_int),
    "dd_solve": ([ctypes.c_void_p, ctypes.POINTER(SolveParams), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dd_solve_noalloc": ([ctypes.c_void_p, ctypes.POINTER(SolveParams), ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dd_create_mg": ([ctypes.c_void_p, ctypes.POINTER(MgParams), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
                     ctypes.c_int),
    "dd_mg_coarse_length": ([ctypes.c_void_p], ctypes.c_size_t),
    "dd_mg_restrict": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dd_mg_prolong": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dd_mg_coarse_apply": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dd_mg_precondition": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dd_server_create": ([ctypes.POINTER(ServerParams), ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "dd_submit": ([ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "dd_poll": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                 ctypes.c_void_p], ctypes.c_int),
    "dd_cancel": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int),
    "dd_server_get_stats": ([ctypes.c_void_p, ctypes.POINTER(ServerStats)], ctypes.c_int),
}


def build(force: bool = False) -> str:
    return _build.build(force=force)


def library_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if needed) the CUDA library; raise if impossible.
    DD_LIBRARY=<path> loads that build instead (e.g. the index-checking one
    from build.py --checked)."""
    global _lib
    if _lib is None:
        path = os.environ.get("DD_LIBRARY") or _build.build()
        L = ctypes.CDLL(path)
        for name, (args, res) in EXPORTS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise DDError(rc, f"{what}: {lib().dd_last_error().decode()}")


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return ctypes.c_void_p(t.ctypes.data)
    assert t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


class Handle:
    _h = None

    def close(self):
        if self._h:
            lib().dd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h


class Lattice(Handle):
    """dims (T, Z, Y, X); block (T, Z, Y, X) Schwarz block / storage tile."""

    def __init__(self, dims, block, antiperiodic: bool = True):
        h = ctypes.c_void_p()
        d = (ctypes.c_int * 4)(*[int(x) for x in dims])
        b = (ctypes.c_int * 4)(*[int(x) for x in block])
        _check(lib().dd_create_lattice(d, b, int(bool(antiperiodic)), ctypes.byref(h)), "dd_create_lattice")
        self._h = h.value
        self.dims, self.block = tuple(dims), tuple(block)
        self.V = int(lib().dd_lattice_volume(self._h))

    def field_bytes(self, prec: int) -> int:
        return int(lib().dd_field_bytes(self._h, prec))

    def new_field(self, prec: int, nrhs: int = 1, device="cuda"):
        import torch
        return torch.zeros(self.field_bytes(prec) * nrhs, dtype=torch.uint8, device=device)

    def pack(self, prec: int, canon_dev, field, nrhs: int = 1, scale: float = 1.0, stream=None):
        """canonical complex128 device tensor (nrhs, V, 4, 3) -> internal field."""
        _check(lib().dd_pack(self._h, prec, _ptr(canon_dev), _ptr(field), nrhs, scale, _stream_ptr(stream)),
               "dd_pack")

    def unpack(self, prec: int, field, canon_dev, nrhs: int = 1, scale: float = 1.0, stream=None):
        _check(lib().dd_unpack(self._h, prec, _ptr(field), _ptr(canon_dev), nrhs, scale, _stream_ptr(stream)),
               "dd_unpack")

    def to_field(self, psi: np.ndarray, prec: int, scale: float = 1.0):
        """numpy canonical spinors (..., V, 4, 3) -> new device field tensor."""
        import torch
        a = np.ascontiguousarray(psi, dtype=np.complex128)
        nrhs = a.size // (12 * self.V)
        dev = torch.from_numpy(a.view(np.float64).reshape(-1)).cuda()
        f = self.new_field(prec, nrhs)
        self.pack(prec, dev, f, nrhs, scale)
        return f

    def from_field(self, field, prec: int, nrhs: int = 1, scale: float = 1.0) -> np.ndarray:
        import torch
        dev = torch.empty(nrhs * self.V * 24, dtype=torch.float64, device=field.device)
        self.unpack(prec, field, dev, nrhs, scale)
        torch.cuda.synchronize()
        out = dev.cpu().numpy().view(np.complex128)
        return out.reshape(nrhs, self.V, 4, 3) if nrhs > 1 else out.reshape(self.V, 4, 3)


class Gauge(Handle):
    def __init__(self, lat: Lattice, links: np.ndarray):
        a = np.ascontiguousarray(links, dtype=np.complex128)
        assert a.size == lat.V * 36
        h = ctypes.c_void_p()
        _check(lib().dd_create_gauge(lat.handle, _ptr(a), ctypes.byref(h)), "dd_create_gauge")
        self._h = h.value
        self.lat = lat


class Op(Handle):
    """Wilson-clover operator; ``prec`` is the Schwarz smoother's storage precision."""

    def __init__(self, gauge: Gauge, c_sw: float = None, m0: float = None, prec: int = F32, clover=None):
        """Either (c_sw, m0): the clover term is built from the gauge field; or
        clover: caller-supplied site blocks A(n) = 4 + m0 + C(n), (V, 2, 6, 6)
        complex (the layout of ``Op.clover()``)."""
        h = ctypes.c_void_p()
        if clover is not None:
            A = np.ascontiguousarray(clover, dtype=np.complex128)
            if A.size != gauge.lat.V * 72:
                raise ValueError("clover must hold V x 2 x 6 x 6 complex entries")
            _check(lib().dd_create_op_clover(gauge.handle, _ptr(A), int(prec), ctypes.byref(h)),
                   "dd_create_op_clover")
        else:
            _check(lib().dd_create_op(gauge.handle, float(c_sw), float(m0), int(prec), ctypes.byref(h)),
                   "dd_create_op")
        self._h = h.value
        self.gauge, self.lat, self.prec = gauge, gauge.lat, prec

    def clover(self) -> np.ndarray:
        """Site blocks A(n) as (V, 2, 6, 6) complex128."""
        out = np.empty((self.lat.V, 2, 6, 6), dtype=np.complex128)
        _check(lib().dd_op_get_clover(self._h, _ptr(out)), "dd_op_get_clover")
        return out

    def apply_D(self, prec: int, inp, out, nrhs: int = 1, stream=None):
        _check(lib().dd_apply_D(self._h, prec, _ptr(inp), _ptr(out), nrhs, _stream_ptr(stream)), "dd_apply_D")

    def sap_smooth(self, b, x, sweeps: int, mr_steps: int, nrhs: int = 1, x_is_zero: bool = True,
                   rhs_tile: int = 0, stream=None):
        p = SapParams(sweeps, mr_steps, int(bool(x_is_zero)), rhs_tile)
        _check(lib().dd_sap_smooth(self._h, ctypes.byref(p), _ptr(b), _ptr(x), nrhs, _stream_ptr(stream)),
               "dd_sap_smooth")

    def solve(self, b, x=None, tol=1e-10, restart=16, max_iter=1000, sweeps=4, mr_steps=4,
              inner_reduction=None, use_x0=False, stream=None, raise_on_notconv=True, mg=None,
              outer_f64=False):
        """Solve D x = b. b: numpy (host) or torch (device) canonical spinors
        (nrhs, V, 4, 3) complex128 or their float64 view. Returns (x, infos).
        outer_f64: IEEE FP64 Krylov basis and true residual also for a
        mixed-precision operator (default: double-float)."""
        if inner_reduction is None:
            inner_reduction = 0.0 if self.prec == F64 else 1e-5
        on_dev = not isinstance(b, np.ndarray)
        b = _as_canonical(b, self.lat.V)
        nrhs = _count_rhs(b, self.lat.V)
        if x is None:
            x = (np.zeros_like(b) if not on_dev else b.new_zeros(b.shape))
        else:
            x = _as_canonical(x, self.lat.V)
            if _count_rhs(x, self.lat.V) != nrhs:
                raise ValueError("x and b hold different numbers of right-hand sides")
        p = SolveParams(tol, restart, max_iter, SapParams(sweeps, mr_steps, 1, 0), inner_reduction,
                        DEVICE if on_dev else HOST, int(bool(use_x0)), mg.handle if mg is not None else None,
                        int(bool(outer_f64)))
        infos = (SolveInfo * nrhs)()
        rc = lib().dd_solve(self._h, ctypes.byref(p), _ptr(b), _ptr(x), nrhs, infos, _stream_ptr(stream))
        if rc != 0 and not (rc == -4 and not raise_on_notconv):
            _check(rc, "dd_solve")
        return x, [i.as_dict() for i in infos]


def sap_smooth_multi(items, sweeps: int, mr_steps: int, x_is_zero: bool = True, rhs_tile: int = 0, stream=None):
    """dd_sap_smooth_multi: items = [(op, b_field, x_field, nrhs), ...], the
    Schwarz smoother of every operator's right-hand sides in one launch per
    colour phase."""
    n = len(items)
    ops = (ctypes.c_void_p * n)(*[op.handle for op, _, _, _ in items])
    nrhs = (ctypes.c_int * n)(*[int(k) for _, _, _, k in items])
    bs = (ctypes.c_void_p * n)(*[_ptr(b).value for _, b, _, _ in items])
    xs = (ctypes.c_void_p * n)(*[_ptr(x).value for _, _, x, _ in items])
    p = SapParams(sweeps, mr_steps, int(bool(x_is_zero)), rhs_tile)
    _check(lib().dd_sap_smooth_multi(n, ops, nrhs, ctypes.byref(p), bs, xs, _stream_ptr(stream)),
           "dd_sap_smooth_multi")


NOALLOC_SCRATCH_BYTES = 64 << 20


def solve_noalloc(op: "Op", b_dev, x_dev, tol=1e-10, restart=16, max_iter=1000, sweeps=4, mr_steps=4,
                  inner_reduction=None, use_x0=False, stream=None):
    """dd_solve_noalloc: one right-hand side, device buffers, no allocation.
    b_dev and x_dev are contiguous CUDA float64/complex128 tensors holding one
    canonical spinor field each. Returns the solve record as a dict."""
    b_dev = _as_canonical(b_dev, op.lat.V)
    x_dev = _as_canonical(x_dev, op.lat.V)
    if isinstance(b_dev, np.ndarray) or isinstance(x_dev, np.ndarray):
        raise TypeError("solve_noalloc takes device tensors")
    if _count_rhs(b_dev, op.lat.V) != 1 or _count_rhs(x_dev, op.lat.V) != 1:
        raise ValueError("solve_noalloc solves exactly one right-hand side")
    if inner_reduction is None:
        inner_reduction = 0.0 if op.prec == F64 else 1e-5
    p = SolveParams(tol, restart, max_iter, SapParams(sweeps, mr_steps, 1, 0), inner_reduction, DEVICE,
                    int(bool(use_x0)))
    info = SolveInfo()
    _check(lib().dd_solve_noalloc(op.handle, ctypes.byref(p), _ptr(b_dev), _ptr(x_dev), ctypes.byref(info),
                                  _stream_ptr(stream)), "dd_solve_noalloc")
    return info.as_dict()


def _as_canonical(a, V: int):
    """Canonical FP64 spinors as complex128 (numpy) or float64/complex128
    (torch, device); float64 numpy arrays are reinterpreted, never converted."""
    if isinstance(a, np.ndarray):
        if a.dtype == np.float64:
            a = a.view(np.complex128)
        if a.dtype != np.complex128 or not a.flags.c_contiguous:
            raise TypeError("host spinors must be C-contiguous complex128 (or their float64 view)")
        return a
    import torch
    if a.dtype not in (torch.float64, torch.complex128) or not a.is_contiguous() or not a.is_cuda:
        raise TypeError("device spinors must be contiguous CUDA float64/complex128 tensors")
    return a


def _count_rhs(a, V: int) -> int:
    reals = a.size * 2 if isinstance(a, np.ndarray) else a.numel() * (2 if a.is_complex() else 1)
    if reals % (24 * V):
        raise ValueError("spinor array size is not a whole number of lattice fields")
    return reals // (24 * V)


class Multigrid(Handle):
    """Two-level preconditioner (dd_create_mg) built from host test vectors
    (N, V, 4, 3) complex128 on the lattice's Schwarz blocks as aggregates."""

    def __init__(self, op: Op, test_vectors, setup_iters=3, coarse_max_iter=24, coarse_tol=0.05, sweeps=4,
                 mr_steps=4):
        tv = np.ascontiguousarray(test_vectors, dtype=np.complex128)
        n = tv.size // (12 * op.lat.V)
        p = MgParams(n, setup_iters, coarse_max_iter, coarse_tol, SapParams(sweeps, mr_steps, 1, 0))
        h = ctypes.c_void_p()
        _check(lib().dd_create_mg(op.handle, ctypes.byref(p), _ptr(tv), ctypes.byref(h)), "dd_create_mg")
        self._h = h.value
        self.op, self.N = op, n
        self.coarse_length = int(lib().dd_mg_coarse_length(self._h))

    def new_coarse(self, device="cuda"):
        import torch
        return torch.zeros(2 * self.coarse_length, dtype=torch.float32, device=device)

    def restrict(self, fine_f32, coarse, stream=None):
        _check(lib().dd_mg_restrict(self._h, _ptr(fine_f32), _ptr(coarse), _stream_ptr(stream)), "dd_mg_restrict")

    def prolong(self, coarse, fine_f32, stream=None):
        _check(lib().dd_mg_prolong(self._h, _ptr(coarse), _ptr(fine_f32), _stream_ptr(stream)), "dd_mg_prolong")

    def coarse_apply(self, cin, cout, stream=None):
        _check(lib().dd_mg_coarse_apply(self._h, _ptr(cin), _ptr(cout), _stream_ptr(stream)), "dd_mg_coarse_apply")

    def precondition(self, r_f32, x_f32, stream=None):
        _check(lib().dd_mg_precondition(self._h, _ptr(r_f32), _ptr(x_f32), _stream_ptr(stream)),
               "dd_mg_precondition")

    @staticmethod
    def coarse_to_numpy(t, nagg: int, N: int) -> np.ndarray:
        import torch
        torch.cuda.synchronize()
        return t.cpu().numpy().view(np.complex64).astype(np.complex128).reshape(nagg, 2, N)

    @staticmethod
    def coarse_from_numpy(c: np.ndarray):
        import torch
        a = np.ascontiguousarray(c, dtype=np.complex64).reshape(-1)
        return torch.from_numpy(a.view(np.float32).copy()).cuda()


class Server(Handle):
    """Continuous-batching solve server (dd_server_*)."""

    def __init__(self, hbm_budget_bytes: int = 0, max_slots: int = 8, max_batch_rhs: int = 16):
        h = ctypes.c_void_p()
        p = ServerParams(hbm_budget_bytes, max_slots, max_batch_rhs)
        _check(lib().dd_server_create(ctypes.byref(p), ctypes.byref(h)), "dd_server_create")
        self._h = h.value
        self._keep = {}

    def submit(self, op: Op, b: np.ndarray, tol=1e-10, restart=16, max_iter=1000, sweeps=4, mr_steps=4,
               inner_reduction=None, mg=None) -> int:
        """Queue a solve; ``mg``: a Multigrid of ``op`` to precondition with
        the two-level method instead of SAP."""
        b = _as_canonical(np.ascontiguousarray(b), op.lat.V)
        nrhs = _count_rhs(b, op.lat.V)
        if inner_reduction is None:
            inner_reduction = 0.0 if op.prec == F64 else 1e-5
        sp = SolveParams(tol, restart, max_iter, SapParams(sweeps, mr_steps, 1, 0), inner_reduction, HOST, 0,
                         mg.handle if mg is not None else None)
        req = Request(op.handle, b.ctypes.data, nrhs, sp)
        t = ctypes.c_uint64()
        _check(lib().dd_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "dd_submit")
        self._keep[t.value] = (op, nrhs, mg)   # the library holds no reference on op or mg
        return t.value

    def poll(self, ticket: int):
        """(state, x or None, infos or None); x/infos once the request has ended."""
        op, nrhs, _ = self._keep[ticket]
        st = ctypes.c_int()
        x = np.empty((nrhs, op.lat.V, 4, 3), dtype=np.complex128)
        infos = (SolveInfo * nrhs)()
        _check(lib().dd_poll(self._h, ticket, ctypes.byref(st), _ptr(x), infos), "dd_poll")
        if st.value in (QUEUED, RUNNING):
            return st.value, None, None
        del self._keep[ticket]
        return st.value, (x[0] if nrhs == 1 else x), [i.as_dict() for i in infos]

    def wait(self, ticket: int, timeout: float = 600.0, interval: float = 0.002):
        import time
        t0 = time.time()
        while True:
            st, x, info = self.poll(ticket)
            if x is not None:
                return st, x, info
            if time.time() - t0 > timeout:
                raise TimeoutError(f"ticket {ticket} still in state {st}")
            time.sleep(interval)

    def cancel(self, ticket: int):
        _check(lib().dd_cancel(self._h, ticket), "dd_cancel")

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().dd_server_get_stats(self._h, ctypes.byref(s)), "dd_server_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}


def version() -> str:
    return lib().dd_version().decode()


def kernel_launches() -> int:
    return int(lib().dd_kernel_launches())


def device_status():
    """Wait for the device; raise DDError if a bounded in-kernel wait expired
    since the previous call (dd_device_status)."""
    _check(lib().dd_device_status(), "dd_device_status")


def release_workspace():
    """dd_release_workspace: free the cached solver workspaces (device and
    pinned host buffers) that finished solves left for reuse."""
    _check(lib().dd_release_workspace(), "dd_release_workspace")


def bench_link_product(method: int, ctas: int = 1216, reps: int = 200):
    """dd_bench_link_product: (ms for `reps` passes, products per pass,
    relative difference from the FP32 CUDA-core method)."""
    ms, diff = ctypes.c_double(), ctypes.c_double()
    _check(lib().dd_bench_link_product(int(method), int(ctas), int(reps), ctypes.byref(ms), ctypes.byref(diff)),
           "dd_bench_link_product")
    return ms.value, ctas * 64, diff.value


def selftest_wait(expire: bool):
    """dd_selftest_wait: the bounded in-kernel wait, completing or expiring."""
    _check(lib().dd_selftest_wait(int(bool(expire))), "dd_selftest_wait")
