"""FP64 CPU oracle for the Wilson-clover SAP-FGMRES path (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package. It shares no code with the GPU library. ``oracle.c`` states every
definition it implements and the paper passage each follows; this wrapper only
compiles it on first use and marshals numpy arrays.

Array conventions (complex128):
  links   (V, 4, 3, 3)   spinor (V, 4, 3)   site matrices (V, 12, 12)
  dims (T, Z, Y, X); block dims (T, Z, Y, X)

Every function here is pinned by a test under ``tests/test_oracle_*.py``
against a property the mathematics fixes (gamma5-hermiticity, the free-field
spectrum in closed form, gauge covariance, the tree-level improvement
condition of the clover term, dense solves); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
        pi, pd = P(i), P(d)
        sig = {
            "or_gamma": ([i, pd], i),
            "or_clover_term": ([pi, pd, d, pd], i),
            "or_site_matrix": ([l, pd, d, pd], i),
            "or_site_inverse": ([l, pd, pd], i),
            "or_apply_D": ([pi, i, pd, pd, pd, pd], i),
            "or_apply_DB": ([pi, i, pi, l, pd, pd, pd, pd], i),
            "or_block_solve": ([pi, i, pi, l, pd, pd, pd, pd, pd, i], i),
            "or_block_colour": ([pi, pi, l], i),
            "or_block_site": ([pi, pi, l, l], l),
            "or_sap": ([pi, i, pi, pd, pd, pd, pd, pd, i, i], i),
            "or_fgmres": ([pi, i, pi, pd, pd, pd, pd, pd, i, d, i, i, i, pd], i),
            "or_apply_D_sites": ([pi, i, pd, d, d, pd, P(l), l, pd], i),
            "or_gram_schmidt": ([l, pd, i, pd, pd], i),
            "or_set_threads": ([i], i),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(d):
    return (ctypes.c_int * 4)(*[int(x) for x in d])


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu = 0..3 for x, y, z, t) or gamma5 (mu = 4), 4x4 complex."""
    out = np.empty((4, 4), dtype=np.complex128)
    if _L().or_gamma(int(mu), _dp(out)) != 0:
        raise ValueError(mu)
    return out


def clover_term(dims, U, c_sw: float) -> np.ndarray:
    """C(n) per site as a (V, 12, 12) matrix (no mass term)."""
    U = _c128(U)
    V = U.shape[0]
    out = np.empty((V, 12, 12), dtype=np.complex128)
    if _L().or_clover_term(_dims(dims), _dp(U), float(c_sw), _dp(out)) != 0:
        raise ValueError("or_clover_term")
    return out


def site_matrix(C, m0: float) -> np.ndarray:
    """A(n) = (4 + m0) + C(n)."""
    C = _c128(C)
    out = np.empty_like(C)
    _L().or_site_matrix(C.shape[0], _dp(C), float(m0), _dp(out))
    return out


def site_inverse(A) -> np.ndarray:
    A = _c128(A)
    out = np.empty_like(A)
    if _L().or_site_inverse(A.shape[0], _dp(A), _dp(out)) != 0:
        raise ValueError("singular site matrix")
    return out


def apply_D_sites(dims, U, c_sw: float, m0: float, psi, sites, antiperiodic: bool = True) -> np.ndarray:
    """(D psi)(n) at the given canonical sites, shape (len(sites), 4, 3); the
    clover term is formed on the fly, so no full-lattice site matrices are
    held (for sampled checks on large lattices)."""
    U = _c128(U)
    psi = _c128(psi)
    st = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(st), 4, 3), dtype=np.complex128)
    rc = _L().or_apply_D_sites(_dims(dims), int(bool(antiperiodic)), _dp(U), float(c_sw), float(m0), _dp(psi),
                               st.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), len(st), _dp(out))
    if rc:
        raise ValueError("or_apply_D_sites")
    return out


def set_threads(n: int) -> int:
    """OpenMP threads for the oracle's parallel loops (n <= 0: unchanged);
    returns the number in effect."""
    return int(_L().or_set_threads(int(n)))


def gram_schmidt(V, w):
    """One modified Gram-Schmidt step as FGMRES takes it: w (complex, n) is
    projected against the rows of V (k x n) in order. Returns (w', h)."""
    V = _c128(V)
    w = _c128(w).reshape(-1).copy()
    k = V.shape[0] if V.ndim == 2 else 0
    h = np.zeros(max(k, 1), dtype=np.complex128)
    if _L().or_gram_schmidt(w.size, _dp(V), k, _dp(w), _dp(h)):
        raise ValueError("or_gram_schmidt")
    return w, h[:k]


class Operator:
    """The Wilson-clover operator D on one gauge field, with its site matrices."""

    def __init__(self, dims, U, c_sw: float, m0: float, antiperiodic: bool = True, C=None):
        self.dims = tuple(int(x) for x in dims)
        self.V = int(np.prod(self.dims))
        self.U = _c128(U)
        self.C = clover_term(self.dims, self.U, c_sw) if C is None else _c128(C)
        self.A = site_matrix(self.C, m0)
        self.Ainv = site_inverse(self.A)
        self.ap = int(bool(antiperiodic))
        self.c_sw, self.m0 = c_sw, m0

    def apply(self, psi) -> np.ndarray:
        psi = _c128(psi).reshape(self.V, 4, 3)
        out = np.empty_like(psi)
        if _L().or_apply_D(_dims(self.dims), self.ap, _dp(self.U), _dp(self.A), _dp(psi), _dp(out)):
            raise ValueError("or_apply_D")
        return out

    def apply_block(self, bdims, block: int, psi) -> np.ndarray:
        """D_B psi on the sites of ``block`` (others of the result are zero)."""
        psi = _c128(psi).reshape(self.V, 4, 3)
        out = np.zeros_like(psi)
        if _L().or_apply_DB(_dims(self.dims), self.ap, _dims(bdims), int(block), _dp(self.U),
                            _dp(self.A), _dp(psi), _dp(out)):
            raise ValueError("or_apply_DB")
        return out

    def block_solve(self, bdims, block: int, r, nmr: int) -> np.ndarray:
        r = _c128(r).reshape(self.V, 4, 3)
        e = np.zeros_like(r)
        if _L().or_block_solve(_dims(self.dims), self.ap, _dims(bdims), int(block), _dp(self.U),
                               _dp(self.A), _dp(self.Ainv), _dp(r), _dp(e), int(nmr)):
            raise ValueError("or_block_solve")
        return e

    def block_sites(self, bdims, block: int) -> np.ndarray:
        vb = int(np.prod(bdims))
        return np.array([_L().or_block_site(_dims(self.dims), _dims(bdims), int(block), k)
                         for k in range(vb)], dtype=np.int64)

    def block_colour(self, bdims, block: int) -> int:
        return int(_L().or_block_colour(_dims(self.dims), _dims(bdims), int(block)))

    def nblocks(self, bdims) -> int:
        return int(np.prod([a // b for a, b in zip(self.dims, bdims)]))

    def sap(self, bdims, b, nsweep: int, nmr: int, x0=None) -> np.ndarray:
        """``nsweep`` red-black Schwarz sweeps from x0 (zero: the preconditioner)."""
        b = _c128(b).reshape(self.V, 4, 3)
        x = np.zeros_like(b) if x0 is None else _c128(x0).reshape(self.V, 4, 3).copy()
        rc = _L().or_sap(_dims(self.dims), self.ap, _dims(bdims), _dp(self.U), _dp(self.A),
                         _dp(self.Ainv), _dp(b), _dp(x), int(nsweep), int(nmr))
        if rc:
            raise ValueError(f"or_sap rc={rc}")
        return x

    def fgmres(self, bdims, b, restart: int, tol: float, max_iter: int, nsweep: int, nmr: int,
               x0=None):
        """FGMRES(restart) preconditioned by SAP. Returns (x, converged, stats)."""
        b = _c128(b).reshape(self.V, 4, 3)
        x = np.zeros_like(b) if x0 is None else _c128(x0).reshape(self.V, 4, 3).copy()
        st = np.zeros(3)
        rc = _L().or_fgmres(_dims(self.dims), self.ap, _dims(bdims), _dp(self.U), _dp(self.A),
                            _dp(self.Ainv), _dp(b), _dp(x), int(restart), float(tol),
                            int(max_iter), int(nsweep), int(nmr), _dp(st))
        if rc < 0:
            raise ValueError(f"or_fgmres rc={rc}")
        return x, rc == 0, dict(iterations=int(st[0]), cycles=int(st[1]), rel_residual=float(st[2]))

    def dense(self) -> np.ndarray:
        """The full (12V x 12V) matrix of D, column j = D e_j."""
        n = 12 * self.V
        M = np.empty((n, n), dtype=np.complex128)
        e = np.zeros(n, dtype=np.complex128)
        for j in range(n):
            e[j] = 1.0
            M[:, j] = self.apply(e).reshape(-1)
            e[j] = 0.0
        return M
