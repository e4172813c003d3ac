"""dd_create_op_clover: an operator built from caller-supplied clover site
blocks A(n) (here a perturbed, still chirality-block-diagonal Hermitian
clover that the library could not have computed itself) against the FP64
oracle given the same blocks; the round trip through Op.clover(); a singular
even-site block is refused."""
import numpy as np
import pytest

import oracle
import paper_1710_07041_gb300 as dd
import synth
from gpu_common import relerr

pytestmark = pytest.mark.gpu

DIMS, BLOCK = (8, 4, 4, 8), (4, 2, 2, 4)


def _blocks(A12):
    """(V, 12, 12) site matrices -> (V, 2, 6, 6) chirality blocks."""
    return np.stack([A12[:, 0:6, 0:6], A12[:, 6:12, 6:12]], axis=1)


@pytest.fixture(scope="module")
def field():
    V = int(np.prod(DIMS))
    U = synth.gauge(DIMS, 0.3, 1, 0.1, 61)
    C = oracle.clover_term(DIMS, U, 1.3)
    # a Hermitian perturbation inside each chirality block
    R = (synth.gaussian(V * 144, 62) * 0.05).reshape(V, 12, 12)
    R[:, 0:6, 6:12] = 0
    R[:, 6:12, 0:6] = 0
    C = C + 0.5 * (R + R.conj().transpose(0, 2, 1))
    lat = dd.Lattice(DIMS, BLOCK)
    gauge = dd.Gauge(lat, U)
    yield V, U, C, lat, gauge
    gauge.close()
    lat.close()


@pytest.mark.parametrize("prec,tol", [(dd.F64, 1e-13), (dd.F32, 1e-6)])
def test_apply_D_with_supplied_clover(field, prec, tol):
    V, U, C, lat, gauge = field
    m0 = -0.05
    ref = oracle.Operator(DIMS, U, 1.3, m0, C=C)
    op = dd.Op(gauge, prec=prec, clover=_blocks(ref.A))
    b = synth.gaussian_spinor(V, 63)
    fin, fout = lat.to_field(b, prec), lat.new_field(prec)
    op.apply_D(prec, fin, fout)
    assert relerr(lat.from_field(fout, prec), ref.apply(b)) <= tol
    # the stored blocks come back (FP64, exactly Hermitian input: bit for bit)
    assert np.max(np.abs(op.clover() - _blocks(ref.A))) <= 1e-14 * np.max(np.abs(ref.A))
    op.close()


def test_sap_and_solve_with_supplied_clover(field):
    V, U, C, lat, gauge = field
    m0 = 0.05
    ref = oracle.Operator(DIMS, U, 1.3, m0, C=C)
    op = dd.Op(gauge, prec=dd.F32, clover=_blocks(ref.A))
    b = synth.gaussian_spinor(V, 64)
    fb, fx = lat.to_field(b, dd.F32), lat.new_field(dd.F32)
    op.sap_smooth(fb, fx, 2, 4)
    assert relerr(lat.from_field(fx, dd.F32), ref.sap(BLOCK, b, 2, 4)) <= 5e-7
    x, info = op.solve(b, tol=1e-10)
    assert relerr(ref.apply(x), b) <= 1e-10
    op.close()


def test_singular_block_refused(field):
    V, U, C, lat, gauge = field
    A = _blocks(oracle.site_matrix(C, 0.1))
    A[0, 1] = 0.0            # canonical site 0 is even: its chirality-1 block is singular
    with pytest.raises(dd.DDError):
        dd.Op(gauge, prec=dd.F32, clover=A)
