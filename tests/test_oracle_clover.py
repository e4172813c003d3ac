"""Pins of the oracle's clover term C(n) and site matrices A(n) = 4 + m0 + C(n).

The clover term's sign and normalisation are a convention that the paper does
not state. The reading taken is the Sheikholeslami-Wohlert term with tree-level
coefficient c_sw = 1 cancelling the O(a) Pauli term of the Wilson operator.
``test_tree_level_improvement`` pins exactly that: in a constant abelian
magnetic field the would-be zero modes of the Wilson operator are lifted by
O(F) at c_sw = 0 and only by O(F^2) at c_sw = 1.
"""
import numpy as np

import oracle
import synth
from test_oracle_operator import gauge_transform


def test_clover_hermitian_chiral_traceless():
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, 0.4, 1, 0.1, seed=31)
    C = oracle.clover_term(dims, U, 1.7)
    assert np.allclose(C, np.conj(np.swapaxes(C, 1, 2)), atol=1e-14)
    g5 = np.kron(oracle.gamma(4), np.eye(3))
    assert np.allclose(C @ g5, g5 @ C, atol=1e-14)
    # block diagonal: no coupling between spins {0,1} and {2,3}
    assert abs(C[:, :6, 6:]).max() < 1e-14
    # spin trace vanishes (tr g_mu g_nu = 0 for mu != nu)
    Cs = C.reshape(-1, 4, 3, 4, 3)
    assert abs(np.einsum("nsasb->nab", Cs)).max() < 1e-13
    assert abs(C).max() > 0.01
    # linear in c_sw
    assert np.allclose(oracle.clover_term(dims, U, 3.4), 2 * C, atol=1e-14)


def test_clover_vanishes_on_unit_gauge():
    dims = (4, 4, 4, 4)
    assert abs(oracle.clover_term(dims, synth.unit_gauge(dims), 1.7)).max() == 0


def test_clover_gauge_covariance():
    dims = (4, 4, 4, 4)
    V = 256
    U = synth.gauge(dims, 0.4, 0, 0.1, seed=32)
    G = synth.su3_field(V, 1.0, seed=33)
    C = oracle.clover_term(dims, U, 1.0)
    Cp = oracle.clover_term(dims, gauge_transform(U, G, dims), 1.0)
    Gb = np.einsum("st,nab->nsatb", np.eye(4), G).reshape(V, 12, 12)
    assert np.allclose(Cp, Gb @ C @ np.conj(np.swapaxes(Gb, 1, 2)), atol=1e-13)


def test_site_inverse():
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, 0.3, 0, 0.1, seed=1)
    C = oracle.clover_term(dims, U, 1.0)
    A = oracle.site_matrix(C, 0.1)
    assert np.allclose(A - C, 4.1 * np.eye(12)[None], atol=1e-15)
    Ai = oracle.site_inverse(A)
    assert abs(A @ Ai - np.eye(12)).max() < 1e-13


def _constant_field(dims, k):
    """U(1) x U(1) constant field F = 2 pi k / (X Y) in the x-y plane, embedded
    as diag(e^{i theta}, e^{-i theta}, 1) in SU(3); every x-y plaquette of
    colour 0 equals e^{iF}."""
    T, Z, Y, X = dims
    F = 2 * np.pi * k / (X * Y)
    U = synth.unit_gauge(dims).reshape(T, Z, Y, X, 4, 3, 3)
    for y in range(Y):
        ph = np.exp(-1j * F * y)
        U[:, :, y, :, 0, 0, 0] = ph
        U[:, :, y, :, 0, 1, 1] = np.conj(ph)
    for x in range(X):
        ph = np.exp(1j * F * Y * x)
        U[:, :, Y - 1, x, 1, 0, 0] = ph
        U[:, :, Y - 1, x, 1, 1, 1] = np.conj(ph)
    return U.reshape(-1, 4, 3, 3), F


def test_tree_level_improvement():
    dims = (2, 2, 8, 8)
    V = int(np.prod(dims))
    U, F = _constant_field(dims, 1)
    idx = np.array([n * 12 + 3 * s for n in range(V) for s in range(4)])  # colour 0
    low = {}
    for c_sw in (0.0, 1.0, -1.0):
        op = oracle.Operator(dims, U, c_sw, 0.0, antiperiodic=False)
        ev = np.linalg.eigvals(op.dense()[np.ix_(idx, idx)])
        low[c_sw] = ev[np.argsort(abs(ev))[:2]]
    # Wilson term alone lifts the two zero modes to about +F/2 (real)
    assert np.allclose(low[0.0].real, F / 2, rtol=0.05) and abs(low[0.0].imag).max() < 1e-10
    # the clover term at c_sw = 1 cancels that O(F) shift
    assert abs(low[1.0]).max() < 0.03 * abs(low[0.0]).min()
    # the opposite sign would double it
    assert np.allclose(low[-1.0].real, 2 * low[0.0].real, rtol=0.05)
