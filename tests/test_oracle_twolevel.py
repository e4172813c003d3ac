"""Pins of the oracle's two-level (aggregation multigrid) preconditioner.

Properties fixed by the construction, none re-typing the oracle's code:
orthonormal interpolation, restriction = prolongation^dagger, the test
vectors lie in range(P), gamma5-hermiticity of the Galerkin coarse operator
(chirality-split aggregates), the Galerkin projection property of an exact
coarse correction, gauge invariance of D_c under covariant test vectors, the coarse GMRES
against a dense solve of D_c (with and without restarts) and, step by step,
against the minimum residual over the Krylov space found by brute force
(which also fixes its stopping rule), and convergence of the two-level
FGMRES to a dense LU solution in fewer steps than the Schwarz
preconditioner alone.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.twolevel import TwoLevel
from test_oracle_operator import gauge_transform

DIMS = (4, 4, 4, 4)
V = 256
CB = (2, 2, 2, 2)


@pytest.fixture(scope="module")
def op():
    U = synth.gauge(DIMS, 0.3, 1, 0.1, seed=81)
    return oracle.Operator(DIMS, U, c_sw=1.0, m0=-0.05)


def _tv(n, seed):
    return np.stack([synth.gaussian_spinor(V, seed + k) for k in range(n)])


def test_interpolation_orthonormal_and_adjoint(op):
    tl = TwoLevel(op, CB, _tv(5, 100))
    for qa in tl.Q:
        for q in qa:
            assert np.allclose(q.conj().T @ q, np.eye(tl.N), atol=1e-13)
    c = synth.gaussian(tl.nagg * 2 * tl.N, 7).reshape(tl.nagg, 2, tl.N)
    r = synth.gaussian_spinor(V, 8)
    assert np.isclose(np.vdot(tl.prolong(c), r), np.vdot(c, tl.restrict(r)), rtol=1e-13)
    assert np.allclose(tl.restrict(tl.prolong(c)), c, atol=1e-13)


def test_test_vectors_in_range_of_P(op):
    tv = _tv(5, 200)
    tl = TwoLevel(op, CB, tv)
    for v in tv:
        assert np.allclose(tl.prolong(tl.restrict(v)), v, atol=1e-12)


def _coarse_dense(tl):
    n = tl.nagg * 2 * tl.N
    M = np.empty((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        M[:, j] = tl.coarse_apply(e).reshape(-1)
    return M


def test_coarse_operator_gamma5_hermitian(op):
    tl = TwoLevel(op, CB, _tv(4, 300))
    M = _coarse_dense(tl)
    g5 = np.tile(np.repeat([1.0, -1.0], tl.N), tl.nagg)
    assert np.allclose(g5[:, None] * M * g5[None, :], M.conj().T, atol=1e-12)


def test_exact_coarse_correction_is_galerkin_projection(op):
    tl = TwoLevel(op, CB, _tv(4, 400))
    M = _coarse_dense(tl)
    r = synth.gaussian_spinor(V, 9)
    ec = np.linalg.solve(M, tl.restrict(r).reshape(-1))
    x = tl.prolong(ec)
    assert np.abs(tl.restrict(r - op.apply(x))).max() < 1e-12 * np.abs(r).max()


def test_coarse_operator_gauge_invariant(op):
    tv = _tv(3, 500)
    G = synth.su3_field(V, 1.0, seed=501)
    opp = oracle.Operator(DIMS, gauge_transform(op.U, G, DIMS), c_sw=1.0, m0=-0.05)
    tvp = np.einsum("nab,knsb->knsa", G, tv)
    M = _coarse_dense(TwoLevel(op, CB, tv))
    Mp = _coarse_dense(TwoLevel(opp, CB, tvp))
    assert np.allclose(M, Mp, atol=1e-12)


@pytest.fixture(scope="module")
def coarse(op):
    tl = TwoLevel(op, CB, _tv(4, 700))
    M = _coarse_dense(tl)
    rhs = synth.gaussian(tl.nagg * 2 * tl.N, 701).reshape(tl.nagg, 2, tl.N)
    return tl, M, rhs


@pytest.mark.parametrize("restart", [200, 7])
def test_coarse_gmres_matches_dense_solve(coarse, restart):
    """Run to 1e-12: one cycle (restart >= dimension) and many short cycles
    (restart 7), so the restart bookkeeping (x accumulated across cycles,
    residual recomputed from D_c) is exercised."""
    tl, M, rhs = coarse
    x = tl.coarse_gmres(rhs, restart=restart, max_iter=2000, tol=1e-12).reshape(-1)
    b = rhs.reshape(-1)
    assert np.linalg.norm(b - M @ x) <= 1e-12 * np.linalg.norm(b) * 1.01
    xs = np.linalg.solve(M, b)
    assert np.linalg.norm(x - xs) <= np.linalg.cond(M) * 1e-12 * np.linalg.norm(xs)


def _krylov_min_residuals(M, b, kmax):
    """min over x in span{b, Mb, ..., M^(k-1) b} of |b - M x|, k = 1..kmax,
    by least squares on the explicit (column-normalised) Krylov matrix."""
    K = [b / np.linalg.norm(b)]
    res = []
    for k in range(1, kmax + 1):
        Kk = np.column_stack(K)
        y, *_ = np.linalg.lstsq(M @ Kk, b, rcond=None)
        res.append(np.linalg.norm(b - M @ (Kk @ y)))
        nxt = M @ K[-1]
        K.append(nxt / np.linalg.norm(nxt))
    return np.array(res)


def test_coarse_gmres_steps_are_krylov_minimisers(coarse):
    """After k steps from zero (no restart) the iterate minimises the
    residual over the k-dimensional Krylov space; one step is the closed form
    x = alpha b, alpha = <M b, b> / <M b, M b>."""
    tl, M, rhs = coarse
    b = rhs.reshape(-1)
    x1 = tl.coarse_gmres(rhs, restart=50, max_iter=1, tol=1e-14).reshape(-1)
    Mb = M @ b
    assert np.allclose(x1, np.vdot(Mb, b) / np.vdot(Mb, Mb).real * b, rtol=1e-12, atol=0)
    rmin = _krylov_min_residuals(M, b, 6)
    for k in range(1, 7):
        xk = tl.coarse_gmres(rhs, restart=50, max_iter=k, tol=1e-14).reshape(-1)
        assert np.isclose(np.linalg.norm(b - M @ xk), rmin[k - 1], rtol=1e-8), k


def test_coarse_gmres_stops_at_first_step_below_tol(coarse):
    """With a loose tolerance the solve stops at the first step whose
    minimal residual reaches tol |b|, neither earlier nor later."""
    tl, M, rhs = coarse
    b = rhs.reshape(-1)
    rmin = _krylov_min_residuals(M, b, 12)
    tol = 0.5 * (rmin[4] + rmin[5]) / np.linalg.norm(b)   # between steps 5 and 6
    x = tl.coarse_gmres(rhs, restart=50, max_iter=100, tol=tol).reshape(-1)
    assert np.isclose(np.linalg.norm(b - M @ x), rmin[5], rtol=1e-8)


def _smoothed_tv(op, block, n, nset, seed):
    tv = np.stack([synth.gaussian_spinor(op.V, seed + k) for k in range(n)])
    for _ in range(nset):   # smooth the test vectors with the Schwarz method
        tv = np.stack([op.sap(block, v, 4, 3) for v in tv])
        tv /= np.linalg.norm(tv.reshape(len(tv), -1), axis=1)[:, None, None, None]
    return tv


MKW = dict(sap_block=CB, sweeps=2, nmr=3, coarse_restart=16, coarse_iter=40, coarse_tol=1e-2)


def test_two_level_fgmres_matches_dense_lu(op):
    b = synth.gaussian_spinor(V, 10)
    tl = TwoLevel(op, CB, _smoothed_tv(op, CB, 6, 3, 600))
    x, its = tl.fgmres(b, restart=16, tol=1e-10, max_iter=200, **MKW)
    D = op.dense()
    assert np.linalg.norm(b.reshape(-1) - D @ x.reshape(-1)) / np.linalg.norm(b) <= 1e-10
    x_lu = np.linalg.solve(D, b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - x_lu) / np.linalg.norm(x_lu) <= np.linalg.cond(D) * 1e-10


def test_two_level_needs_fewer_iterations_than_sap():
    dims = (8, 4, 4, 4)
    op8 = oracle.Operator(dims, synth.gauge(dims, 0.3, 1, 0.1, seed=81), c_sw=1.0, m0=-0.05)
    b = synth.gaussian_spinor(op8.V, 10)
    tl = TwoLevel(op8, CB, _smoothed_tv(op8, CB, 8, 4, 600))
    x, its = tl.fgmres(b, restart=16, tol=1e-10, max_iter=300, **MKW)
    assert np.linalg.norm(b - op8.apply(x)) / np.linalg.norm(b) <= 1e-10
    _, ok, st = op8.fgmres(CB, b, 16, 1e-10, 500, 2, 3)
    assert ok and its <= 0.6 * st["iterations"], (its, st["iterations"])
