"""Pins of the oracle's Schwarz method, block MR and FGMRES.

Sec. 3.1 of the paper names "the MR inversion within a domain" (Table 1) and
"the entire Schwarz method" (Table 2) without defining them. The oracle's
reading (red-black multiplicative Schwarz, even-odd Schur complement on odd
sites, minimal-residual steps, right-preconditioned FGMRES) is pinned here by
dense linear algebra on tiny lattices and by exact invariances:
  * MR run to convergence reproduces the dense block inverse D_B^-1,
  * the even-site block residual vanishes for every MR step count (exact
    reconstruction), and one MR step is the least-squares optimum on span{bhat},
  * one sweep with exact block solves equals K0 b + K1 (b - D K0 b),
  * complex homogeneity and gauge covariance of the fixed-step smoother,
  * FGMRES reaches a true residual of 1e-10 and agrees with a dense LU solve,
    and on the free field with the exact solution built in momentum space.
"""
import numpy as np
import pytest

import oracle
import synth
from test_oracle_operator import gauge_transform

DIMS = (4, 4, 4, 4)
V = 256
BD = (2, 2, 2, 2)


@pytest.fixture(scope="module")
def op(small_gauge):
    return oracle.Operator(DIMS, small_gauge, c_sw=1.0, m0=0.1)


def _block_dense(op, bd, blk):
    """D_B on the block's sites as a dense (12 vb) x (12 vb) matrix."""
    sites = op.block_sites(bd, blk)
    n = 12 * len(sites)
    M = np.empty((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros((V, 12), dtype=complex)
        e[sites[j // 12], j % 12] = 1
        M[:, j] = op.apply_block(bd, blk, e).reshape(V, 12)[sites].reshape(-1)
    return sites, M


def _parity(sites):
    T, Z, Y, X = DIMS
    x = sites % X
    y = (sites // X) % Y
    z = (sites // (X * Y)) % Z
    t = sites // (X * Y * Z)
    return (x + y + z + t) % 2


def test_block_operator_drops_outgoing_hops(op):
    """D_B equals D restricted to the block with hops to outside sites removed:
    applying D to a vector supported on the block and restricting to it gives D_B."""
    r = synth.gaussian_spinor(V, 3)
    for blk in (0, 5):
        sites = op.block_sites(BD, blk)
        v = np.zeros_like(r)
        v[sites] = r[sites]
        full = op.apply(v)[sites]
        blockwise = op.apply_block(BD, blk, v)[sites]
        assert np.allclose(full, blockwise, atol=1e-14)


def test_mr_to_convergence_is_dense_block_inverse(op):
    r = synth.gaussian_spinor(V, 4)
    for blk in (0, 9):
        sites, M = _block_dense(op, BD, blk)
        e = op.block_solve(BD, blk, r, nmr=200)
        want = np.linalg.solve(M, r[sites].reshape(-1))
        got = e[sites].reshape(-1)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-10


@pytest.mark.parametrize("nmr", [0, 1, 2, 5])
def test_even_residual_exact_and_mr_optimal(op, nmr):
    r = synth.gaussian_spinor(V, 5)
    blk = 3
    sites, M = _block_dense(op, BD, blk)
    par = np.repeat(_parity(sites), 12)
    ev, od = par == 0, par == 1
    rb = r[sites].reshape(-1)
    e = op.block_solve(BD, blk, r, nmr=nmr)[sites].reshape(-1)
    res = rb - M @ e
    assert np.linalg.norm(res[ev]) < 1e-13 * np.linalg.norm(rb)
    # odd residual equals the Schur residual bhat - Dhat e_o
    Dee, Deo, Doe, Doo = M[np.ix_(ev, ev)], M[np.ix_(ev, od)], M[np.ix_(od, ev)], M[np.ix_(od, od)]
    Dhat = Doo - Doe @ np.linalg.solve(Dee, Deo)
    bhat = rb[od] - Doe @ np.linalg.solve(Dee, rb[ev])
    assert np.allclose(res[od], bhat - Dhat @ e[od], atol=1e-12)
    if nmr == 1:
        alpha = np.linalg.lstsq((Dhat @ bhat)[:, None], bhat, rcond=None)[0][0]
        assert np.allclose(e[od], alpha * bhat, atol=1e-13)


def test_mr_residual_decreases(op):
    r = synth.gaussian_spinor(V, 6)
    blk = 2
    sites, M = _block_dense(op, BD, blk)
    rb = r[sites].reshape(-1)
    norms = [np.linalg.norm(rb - M @ op.block_solve(BD, blk, r, nmr=k)[sites].reshape(-1))
             for k in range(6)]
    assert all(b < a for a, b in zip(norms, norms[1:]))


def test_block_colouring_is_red_black(op):
    nb = op.nblocks(BD)
    col = np.array([op.block_colour(BD, b) for b in range(nb)])
    assert col.sum() == nb // 2
    # neighbouring blocks (differing by one block step) have opposite colours
    T, Z, Y, X = [a // b for a, b in zip(DIMS, BD)]
    c = col.reshape(T, Z, Y, X)
    for ax in range(4):
        assert np.all(c != np.roll(c, 1, axis=ax))


def test_one_sweep_with_exact_block_solves_matches_dense_formula(op):
    """x = K0 b + K1 (b - D K0 b), K_c = sum over colour-c blocks of I_B D_B^-1 I_B^T."""
    b = synth.gaussian_spinor(V, 7).reshape(V, 12)
    D = op.dense()
    nb = op.nblocks(BD)
    K = [np.zeros((12 * V, 12 * V), dtype=complex) for _ in range(2)]
    for blk in range(nb):
        sites, M = _block_dense(op, BD, blk)
        idx = (sites[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)
        K[op.block_colour(BD, blk)][np.ix_(idx, idx)] = np.linalg.inv(M)
    bv = b.reshape(-1)
    x0 = K[0] @ bv
    want = x0 + K[1] @ (bv - D @ x0)
    got = op.sap(BD, b, nsweep=1, nmr=200).reshape(-1)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-10


def test_sweeps_compose(op):
    b = synth.gaussian_spinor(V, 8)
    x1 = op.sap(BD, b, nsweep=1, nmr=3)
    x2 = op.sap(BD, b, nsweep=2, nmr=3)
    assert np.allclose(op.sap(BD, b, nsweep=1, nmr=3, x0=x1), x2, atol=1e-14)


def test_sap_complex_homogeneity(op):
    b = synth.gaussian_spinor(V, 9)
    c = 0.37 - 2.1j
    x = op.sap(BD, b, 4, 3)
    assert np.allclose(op.sap(BD, c * b, 4, 3), c * x, atol=1e-13)


def test_sap_and_fgmres_gauge_covariance(small_gauge):
    G = synth.su3_field(V, 1.0, seed=44)
    Up = gauge_transform(small_gauge, G, DIMS)
    op = oracle.Operator(DIMS, small_gauge, 1.0, 0.1)
    opp = oracle.Operator(DIMS, Up, 1.0, 0.1)
    b = synth.gaussian_spinor(V, 2)
    Gb = np.einsum("nab,nsb->nsa", G, b)
    Gx = lambda x: np.einsum("nab,nsb->nsa", G, x)
    x = op.sap(BD, b, 4, 3)
    assert np.linalg.norm(opp.sap(BD, Gb, 4, 3) - Gx(x)) / np.linalg.norm(x) < 1e-12
    xs, ok, _ = op.fgmres(BD, b, 16, 1e-10, 200, 4, 3)
    xps, okp, _ = opp.fgmres(BD, Gb, 16, 1e-10, 200, 4, 3)
    assert ok and okp
    assert np.linalg.norm(xps - Gx(xs)) / np.linalg.norm(xs) < 1e-9


def test_fgmres_matches_dense_lu(op):
    """Plain FP64 workload on 4^4: true residual <= 1e-10 and agreement with LU."""
    b = synth.gaussian_spinor(V, 2)
    D = op.dense()
    x_lu = np.linalg.solve(D, b.reshape(-1))
    x, ok, st = op.fgmres(BD, b, restart=16, tol=1e-10, max_iter=500, nsweep=4, nmr=3)
    assert ok and st["rel_residual"] <= 1e-10
    true_res = np.linalg.norm(b.reshape(-1) - D @ x.reshape(-1)) / np.linalg.norm(b)
    assert true_res <= 1e-10
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(x.reshape(-1) - x_lu) / np.linalg.norm(x_lu) <= kappa * 1e-10


def test_fgmres_max_iter_and_zero_rhs(op):
    b = synth.gaussian_spinor(V, 2)
    x, ok, st = op.fgmres(BD, b, restart=4, tol=1e-14, max_iter=2, nsweep=1, nmr=1)
    assert not ok and st["iterations"] == 2 and 0 < st["rel_residual"] < 1
    x, ok, st = op.fgmres(BD, np.zeros_like(b), 16, 1e-10, 10, 4, 3)
    assert ok and not x.any()


def test_gram_schmidt_step_is_orthogonal_projection():
    """The oracle's Arnoldi projection step (the one or_fgmres uses): against
    an orthonormal basis Q it returns h = Q^dagger w and w - Q h, which is
    orthogonal to every basis vector (closed form of the projection)."""
    rng = np.random.default_rng(5)
    n, k = 120, 6
    Q, _ = np.linalg.qr(rng.normal(size=(n, k)) + 1j * rng.normal(size=(n, k)))
    w = rng.normal(size=n) + 1j * rng.normal(size=n)
    w2, h = oracle.gram_schmidt(Q.T.copy(), w)
    assert np.allclose(h, Q.conj().T @ w, rtol=0, atol=1e-13)
    assert np.allclose(w2, w - Q @ (Q.conj().T @ w), rtol=0, atol=1e-13)
    assert np.abs(Q.conj().T @ w2).max() < 1e-13
    w0, h0 = oracle.gram_schmidt(np.zeros((0, n), dtype=complex), w)
    assert h0.size == 0 and np.array_equal(w0, w)


def test_free_field_solve_matches_momentum_space():
    """U = 1 on 8 x 4^3 (antiperiodic time): the SAP-FGMRES solution equals
    the exact solution built in momentum space, independent of any dense
    solve. With the time twist e^{i pi t / T}, a field is a sum of plane waves
    e^{ipn} with p_mu = 2 pi k / L_mu (space) and p_t = (2k + 1) pi / T, and on
    each the operator is the 12 x 12 matrix
    D(p) = (m0 + sum_mu (1 - cos p_mu)) + i sum_mu (g_mu x 1_3) sin p_mu
    (the closed form pinned by test_free_field_plane_waves). D(p) is normal, so
    the condition number of D is the ratio of the largest and smallest
    |M(p) +- i |sin p||; the solution error is bounded by it times 1e-10."""
    dims = (8, 4, 4, 4)
    T, Z, Y, X = dims
    Vf = T * Z * Y * X
    m0 = 0.1
    opf = oracle.Operator(dims, synth.unit_gauge(dims), c_sw=1.0, m0=m0)
    b = synth.gaussian_spinor(Vf, 91).reshape(T, Z, Y, X, 12)
    t = np.arange(T).reshape(T, 1, 1, 1, 1)
    twist = np.exp(1j * np.pi * t / T)
    c = np.fft.fftn(b / twist, axes=(0, 1, 2, 3))   # plane-wave coefficients x V
    g = [np.kron(oracle.gamma(mu), np.eye(3)) for mu in range(4)]
    kt, kz, ky, kx = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    p = [2 * np.pi * kx / X, 2 * np.pi * ky / Y, 2 * np.pi * kz / Z, (2 * kt + 1) * np.pi / T]
    M = m0 + sum(1 - np.cos(q) for q in p)
    s2 = sum(np.sin(q) ** 2 for q in p)
    Dp = M[..., None, None] * np.eye(12) + 1j * sum(np.sin(p[mu])[..., None, None] * g[mu] for mu in range(4))
    xt = np.linalg.solve(Dp, c[..., None])[..., 0]
    x_exact = (np.fft.ifftn(xt, axes=(0, 1, 2, 3)) * twist).reshape(Vf, 12)
    b = b.reshape(Vf, 12)
    # the momentum-space construction is the inverse of the oracle's D
    assert np.linalg.norm(opf.apply(x_exact).reshape(Vf, 12) - b) / np.linalg.norm(b) < 1e-13
    x, ok, st = opf.fgmres((2, 2, 2, 2), b, restart=16, tol=1e-10, max_iter=500, nsweep=4, nmr=3)
    assert ok and st["rel_residual"] <= 1e-10
    sv = np.sqrt(M ** 2 + s2)
    kappa = sv.max() / sv.min()
    err = np.linalg.norm(x.reshape(Vf, 12) - x_exact) / np.linalg.norm(x_exact)
    assert err <= kappa * 1e-10
