"""Seeded synthetic inputs (gauge links, right-hand sides, gauge transforms).

Input preparation only: nothing here computes the Dirac operator, the clover
term, the Schwarz smoother or the Krylov solver. The FP64 oracle and the GPU
library both receive these arrays unchanged. The C source (``synth.c``) states
the recipes; this wrapper compiles it on first use and returns numpy arrays.

Array conventions (complex128):
  links   (V, 4, 3, 3)  U_mu(n), mu = 0:x 1:y 2:z 3:t, row-major colour matrix
  spinor  (V, 4, 3)     spin-major, colour minor
  dims    (T, Z, Y, X); site n = x + X*(y + Y*(z + Z*t))
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_SO = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``_build/libsynth.so`` (gcc, OpenMP)."""
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
        d = ctypes.c_double
        lib.synth_gauge.argtypes = [P(ctypes.c_int), d, ctypes.c_int, d, ctypes.c_uint64, P(d)]
        lib.synth_su3_field.argtypes = [ctypes.c_long, d, ctypes.c_uint64, P(d)]
        lib.synth_gaussian.argtypes = [ctypes.c_long, ctypes.c_uint64, P(d)]
        lib.synth_z2.argtypes = [ctypes.c_long, ctypes.c_uint64, P(d)]
        lib.synth_uniform.argtypes = [ctypes.c_long, ctypes.c_uint64, P(d)]
        for f in (lib.synth_gauge, lib.synth_su3_field, lib.synth_gaussian, lib.synth_z2,
                  lib.synth_uniform):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def volume(dims) -> int:
    return int(np.prod(dims))


def gauge(dims, eps: float, n_stout: int = 0, rho: float = 0.1, seed: int = 1) -> np.ndarray:
    """Links U = exp(i eps H) per (site, mu), then ``n_stout`` stout steps of weight rho."""
    V = volume(dims)
    out = np.empty((V, 4, 3, 3), dtype=np.complex128)
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    rc = _L().synth_gauge(d, float(eps), int(n_stout), float(rho), int(seed), _dp(out))
    if rc != 0:
        raise ValueError("synth_gauge failed")
    return out


def unit_gauge(dims) -> np.ndarray:
    V = volume(dims)
    out = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    out[:, :, 0, 0] = out[:, :, 1, 1] = out[:, :, 2, 2] = 1.0
    return out


def su3_field(V: int, eps: float, seed: int) -> np.ndarray:
    """One random SU(3) matrix per site, exp(i eps H): a gauge transformation."""
    out = np.empty((V, 3, 3), dtype=np.complex128)
    if _L().synth_su3_field(int(V), float(eps), int(seed), _dp(out)) != 0:
        raise ValueError("synth_su3_field failed")
    return out


def gaussian(n_complex: int, seed: int) -> np.ndarray:
    """``n_complex`` complex entries with N(0,1) real and imaginary parts."""
    out = np.empty(n_complex, dtype=np.complex128)
    if _L().synth_gaussian(2 * int(n_complex), int(seed), _dp(out)) != 0:
        raise ValueError("synth_gaussian failed")
    return out


def gaussian_spinor(V: int, seed: int) -> np.ndarray:
    return gaussian(12 * V, seed).reshape(V, 4, 3)


def z2_spinor(V: int, seed: int) -> np.ndarray:
    """Complex Z2 noise: every component (+-1 +- i)/sqrt(2)."""
    out = np.empty(12 * V, dtype=np.complex128)
    if _L().synth_z2(12 * int(V), int(seed), _dp(out)) != 0:
        raise ValueError("synth_z2 failed")
    return out.reshape(V, 4, 3)


def point_source(V: int, spin: int, colour: int, site: int = 0) -> np.ndarray:
    out = np.zeros((V, 4, 3), dtype=np.complex128)
    out[site, spin, colour] = 1.0
    return out


def uniform(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _L().synth_uniform(int(n), int(seed), _dp(out))
    return out


# Workload recipes (lattice, gauge smoothing, operator and solver parameters).
# dims are (T, Z, Y, X); block is the Schwarz block (T, Z, Y, X).
WORKLOADS = {
    "wilson_clover_4^4_fp64": dict(
        dims=(4, 4, 4, 4), eps=0.3, n_stout=0, rho=0.1, c_sw=1.0, m0=0.1,
        gauge_seed=1, rhs_seed=2, block=(2, 2, 2, 2), sweeps=4, mr_steps=3, restart=16),
    "sap_fgmres_64x32^3_fp32": dict(
        dims=(64, 32, 32, 32), eps=0.25, n_stout=2, rho=0.1, c_sw=1.7, m0=-0.02,
        gauge_seed=21, rhs_seed=22, block=(4, 4, 4, 4), sweeps=4, mr_steps=4, restart=16),
    "sap_fgmres_96x48^3_mixed": dict(
        dims=(96, 48, 48, 48), eps=0.2, n_stout=3, rho=0.1, c_sw=1.7, m0=0.0,
        gauge_seed=31, rhs_seed=32, block=(4, 4, 4, 4), sweeps=4, mr_steps=4, restart=32),
    # small case of the 64x32^3 workload for profiler captures (~1.8 GB on the device)
    "profile_32x32x16x16_fp32": dict(
        dims=(32, 32, 16, 16), eps=0.25, n_stout=2, rho=0.1, c_sw=1.7, m0=-0.02,
        gauge_seed=21, rhs_seed=22, block=(4, 4, 4, 4), sweeps=4, mr_steps=4, restart=16),
    "batched_48^3x96_24rhs": dict(
        dims=(96, 48, 48, 48), eps=0.2, n_stout=3, rho=0.1, c_sw=1.7, m0=-0.02,
        gauge_seed=41, rhs_seed=42, block=(4, 4, 4, 4), sweeps=4, mr_steps=4, restart=16),
}
