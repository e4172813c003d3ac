"""Pins of the FP64 oracle's gamma matrices and Wilson-clover operator.

The paper (Sec. 1) only names "the discretized form of the Dirac equation";
these tests fix the oracle's reading of it by properties the mathematics fixes,
none of which re-types the oracle's formula:
  * Clifford algebra and chirality of the gamma matrices,
  * gamma5-hermiticity  g5 D g5 = D^dagger  on a smeared random gauge field,
  * the free-field plane-wave spectrum in closed form (antiperiodic time),
  * gauge covariance under a random SU(3) transformation.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


def test_gamma_clifford_and_chirality():
    g = [oracle.gamma(mu) for mu in range(4)]
    for mu, nu in itertools.product(range(4), repeat=2):
        ac = g[mu] @ g[nu] + g[nu] @ g[mu]
        assert np.allclose(ac, 2 * np.eye(4) * (mu == nu), atol=1e-15)
    for m in g:
        assert np.allclose(m, m.conj().T)
    g5 = oracle.gamma(4)
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3])
    # chiral basis: g5 diagonal with two +1 then two -1
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


def _g5(v):
    g5 = oracle.gamma(4)
    return np.einsum("st,nta->nsa", g5, v)


@pytest.mark.parametrize("dims,n_stout", [((4, 4, 4, 4), 0), ((8, 4, 4, 4), 2)])
def test_gamma5_hermiticity(dims, n_stout):
    V = int(np.prod(dims))
    U = synth.gauge(dims, 0.3, n_stout, 0.1, seed=11)
    op = oracle.Operator(dims, U, c_sw=1.7, m0=-0.02)
    x = synth.gaussian_spinor(V, 12)
    y = synth.gaussian_spinor(V, 13)
    lhs = np.vdot(y, _g5(op.apply(_g5(x))))
    rhs = np.vdot(op.apply(y), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 4, 4, 4)])
def test_free_field_plane_waves(dims):
    """U = 1: D e^{ipn} u = e^{ipn} D(p) u with
    D(p) = m0 + sum_mu (1 - cos p_mu) + i sum_mu g_mu sin p_mu,
    p_mu = 2 pi k / L (space), p_t = (2k + 1) pi / T (antiperiodic time).
    D(p) - M(p) is anti-Hermitian and squares to -sum sin^2 p (convention-free),
    and equals i sum g_mu sin p_mu for the oracle's own (pinned) gammas."""
    T, Z, Y, X = dims
    V = T * Z * Y * X
    m0 = 0.1
    op = oracle.Operator(dims, synth.unit_gauge(dims), c_sw=1.0, m0=m0)
    assert abs(op.C).max() == 0.0
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    g = [oracle.gamma(mu) for mu in range(4)]
    for kt, kz, ky, kx in itertools.product(range(T), range(Z), range(Y), range(X)):
        p = np.array([2 * np.pi * kx / X, 2 * np.pi * ky / Y, 2 * np.pi * kz / Z,
                      (2 * kt + 1) * np.pi / T])
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t)).reshape(V)
        Dp = np.empty((12, 12), dtype=complex)
        for j in range(12):
            psi = np.zeros((V, 12), dtype=complex)
            psi[:, j] = phase
            out = op.apply(psi).reshape(V, 12)
            Dp[:, j] = out[0]
            assert np.allclose(out, phase[:, None] * out[0][None, :], atol=1e-12)
        M = m0 + np.sum(1 - np.cos(p))
        K = Dp - M * np.eye(12)
        assert np.allclose(K, -K.conj().T, atol=1e-12)
        assert np.allclose(K @ K, -np.sum(np.sin(p) ** 2) * np.eye(12), atol=1e-12)
        want = 1j * sum(np.kron(g[mu], np.eye(3)) * np.sin(p[mu]) for mu in range(4))
        assert np.allclose(K, want, atol=1e-12)


def gauge_transform(U, G, dims):
    """U'_mu(n) = G(n) U_mu(n) G(n+mu)^dagger."""
    T, Z, Y, X = dims
    Gl = G.reshape(T, Z, Y, X, 3, 3)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}
    Up = np.empty_like(U).reshape(T, Z, Y, X, 4, 3, 3)
    Ul = U.reshape(T, Z, Y, X, 4, 3, 3)
    for mu in range(4):
        Gs = np.roll(Gl, -1, axis=axes[mu])
        Up[..., mu, :, :] = Gl @ Ul[..., mu, :, :] @ np.conj(np.swapaxes(Gs, -1, -2))
    return Up.reshape(U.shape)


def test_gauge_covariance_of_D():
    dims = (4, 4, 4, 8)
    V = int(np.prod(dims))
    U = synth.gauge(dims, 0.3, 1, 0.1, seed=21)
    G = synth.su3_field(V, 1.0, seed=22)
    Up = gauge_transform(U, G, dims)
    psi = synth.gaussian_spinor(V, 23)
    op = oracle.Operator(dims, U, c_sw=1.7, m0=0.05)
    opp = oracle.Operator(dims, Up, c_sw=1.7, m0=0.05)
    Gpsi = np.einsum("nab,nsb->nsa", G, psi)
    lhs = opp.apply(Gpsi)
    rhs = np.einsum("nab,nsb->nsa", G, op.apply(psi))
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-12


def test_sampled_sites_equal_full_operator():
    """The per-site evaluation used for large lattices equals the full D."""
    dims = (8, 4, 4, 4)
    V = int(np.prod(dims))
    U = synth.gauge(dims, 0.3, 1, 0.1, seed=71)
    psi = synth.gaussian_spinor(V, 72)
    full = oracle.Operator(dims, U, c_sw=1.7, m0=-0.03).apply(psi)
    sites = np.array([0, 1, 17, 100, V - 1, 333])
    part = oracle.apply_D_sites(dims, U, 1.7, -0.03, psi, sites)
    assert np.allclose(part, full[sites], atol=1e-14, rtol=0)
