"""Input generator: links are SU(3), smearing smooths, streams are seeded."""
import numpy as np

import synth


def _plaquette(U, dims):
    T, Z, Y, X = dims
    L = U.reshape(T, Z, Y, X, 4, 3, 3)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Umu, Unu = L[..., mu, :, :], L[..., nu, :, :]
            Unu_xmu = np.roll(Unu, -1, axis=axes[mu])
            Umu_xnu = np.roll(Umu, -1, axis=axes[nu])
            P = Umu @ Unu_xmu @ np.conj(np.swapaxes(Umu_xnu, -1, -2)) @ np.conj(np.swapaxes(Unu, -1, -2))
            tot += np.trace(P, axis1=-2, axis2=-1).real.mean() / 3
    return tot / 6


def test_links_are_su3_after_exp_and_stout():
    for n_stout in (0, 2):
        U = synth.gauge((4, 4, 4, 8), 0.3, n_stout, 0.1, seed=7)
        uu = np.einsum("nmji,nmjk->nmik", U.conj(), U)
        assert abs(uu - np.eye(3)).max() < 1e-13
        assert abs(np.linalg.det(U) - 1).max() < 1e-13


def test_stout_raises_plaquette():
    dims = (4, 4, 4, 4)
    p = [_plaquette(synth.gauge(dims, 0.5, s, 0.1, seed=3), dims) for s in range(3)]
    assert p[0] < p[1] < p[2] < 1.0


def test_small_eps_is_near_identity():
    U = synth.gauge((2, 2, 2, 2), 1e-6, 0, 0.1, seed=1)
    assert abs(U - np.eye(3)).max() < 1e-5


def test_streams_are_seeded():
    a = synth.gaussian(1000, 5)
    assert np.array_equal(a, synth.gaussian(1000, 5))
    assert not np.array_equal(a, synth.gaussian(1000, 6))
    g = synth.gaussian(200000, 9)
    assert abs(g.real.mean()) < 0.01 and abs(g.real.std() - 1) < 0.01 and abs(g.imag.std() - 1) < 0.01
    z = synth.z2_spinor(100, 4)
    assert np.allclose(abs(z.real), 2 ** -0.5) and np.allclose(abs(z.imag), 2 ** -0.5)
    u = synth.uniform(10000, 3)
    assert u.min() > 0 and u.max() <= 1 and abs(u.mean() - 0.5) < 0.02
