"""Shared set-up of the GPU parity tests: the same seeded inputs go to the
CUDA library (through the C ABI) and to the FP64 oracle."""
import numpy as np

import oracle
import paper_1710_07041_gb300 as dd
import synth


def relerr(a, b):
    return float(np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1)))


def worst_site(a, b):
    """Largest per-site error against the RMS site norm of b: max_n |a_n - b_n|
    / sqrt(mean_n |b_n|^2) over spinor sites (arrays (..., 4, 3)). A single
    wrong site among thousands hardly moves the relative L2 error but shows
    here at full size."""
    d = np.linalg.norm((a - b).reshape(-1, 12), axis=1)
    ref = np.sqrt(np.mean(np.linalg.norm(b.reshape(-1, 12), axis=1) ** 2))
    return float(d.max() / ref)


class Setup:
    """A lattice, gauge field and operator on both sides."""

    def __init__(self, dims, block, eps=0.3, n_stout=0, c_sw=1.0, m0=0.1, prec=dd.F32, seed=1,
                 antiperiodic=True, U=None):
        self.dims, self.block = tuple(dims), tuple(block)
        self.V = int(np.prod(dims))
        self.U = synth.gauge(dims, eps, n_stout, 0.1, seed) if U is None else U
        self.lat = dd.Lattice(dims, block, antiperiodic)
        self.gauge = dd.Gauge(self.lat, self.U)
        self.op = dd.Op(self.gauge, c_sw, m0, prec)
        self.ref = oracle.Operator(dims, self.U, c_sw, m0, antiperiodic)
        self.c_sw, self.m0, self.prec = c_sw, m0, prec

    def close(self):
        self.op.close()
        self.gauge.close()
        self.lat.close()
