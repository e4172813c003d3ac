"""GPU parity of the two-level multigrid against the FP64 oracle
(oracle/twolevel.py) on the same seeded test vectors, and the two-level
SAP-FGMRES solve (true residual by the oracle's operator, fewer iterations
than the Schwarz preconditioner alone).

The library keeps the interpolation P and the coarse operator D_c in FP16
(each entry rounded to a relative 2^-11 = 4.9e-4, RMS about 2.8e-4) with FP32
sums, and assembles D_c from the rounded P. Bounds, as relative L2 errors
against the oracle's unrounded FP64 P: 2e-3 for restriction and
prolongation (one factor of P: ~2.8e-4 expected) and for the coarse operator
(two factors of P plus the rounding of D_c: ~6e-4 expected); 5e-3 for a
whole preconditioner application, whose 12 coarse GMRES steps run on the
rounded operator."""
import numpy as np
import pytest

import paper_1710_07041_gb300 as dd
import synth
from gpu_common import Setup, relerr
from oracle.twolevel import TwoLevel

pytestmark = pytest.mark.gpu

DIMS, BLOCK = (8, 8, 8, 8), (4, 4, 4, 4)


@pytest.fixture(scope="module")
def mgsetup():
    s = Setup(DIMS, BLOCK, eps=0.3, n_stout=1, c_sw=1.0, m0=-0.05, prec=dd.F32, seed=91)
    tv = np.stack([synth.gaussian_spinor(s.V, 900 + k) for k in range(6)])
    mg = dd.Multigrid(s.op, tv, setup_iters=0, coarse_max_iter=12, coarse_tol=0.0, sweeps=2, mr_steps=3)
    tl = TwoLevel(s.ref, BLOCK, tv)
    yield s, mg, tl
    mg.close()
    s.close()


def test_restrict_prolong_match_oracle(mgsetup):
    s, mg, tl = mgsetup
    r = synth.gaussian_spinor(s.V, 901)
    rf = s.lat.to_field(r, dd.F32)
    c = mg.new_coarse()
    mg.restrict(rf, c)
    got = dd.Multigrid.coarse_to_numpy(c, tl.nagg, tl.N)
    r32 = s.lat.from_field(rf, dd.F32)
    err = relerr(got, tl.restrict(r32))
    print(f"restrict relerr {err:.3e}")
    assert err <= 2e-3
    cc = synth.gaussian(tl.nagg * 2 * tl.N, 902).reshape(tl.nagg, 2, tl.N)
    xf = s.lat.new_field(dd.F32)
    mg.prolong(dd.Multigrid.coarse_from_numpy(cc), xf)
    x = s.lat.from_field(xf, dd.F32)
    err = relerr(x, tl.prolong(cc.astype(np.complex64)))
    print(f"prolong relerr {err:.3e}")
    assert err <= 2e-3


def test_coarse_operator_matches_galerkin(mgsetup):
    s, mg, tl = mgsetup
    cc = synth.gaussian(tl.nagg * 2 * tl.N, 903).reshape(tl.nagg, 2, tl.N).astype(np.complex64)
    out = mg.new_coarse()
    mg.coarse_apply(dd.Multigrid.coarse_from_numpy(cc), out)
    got = dd.Multigrid.coarse_to_numpy(out, tl.nagg, tl.N)
    err = relerr(got, tl.coarse_apply(cc))
    print(f"coarse apply relerr {err:.3e}")
    assert err <= 2e-3


def test_preconditioner_matches_oracle(mgsetup):
    s, mg, tl = mgsetup
    r = synth.gaussian_spinor(s.V, 904)
    rf = s.lat.to_field(r, dd.F32)
    xf = s.lat.new_field(dd.F32)
    mg.precondition(rf, xf)
    got = s.lat.from_field(xf, dd.F32)
    want = tl.precondition(s.lat.from_field(rf, dd.F32), BLOCK, sweeps=2, nmr=3, coarse_restart=12,
                           coarse_iter=12, coarse_tol=0.0)
    err = relerr(got, want)
    print(f"preconditioner relerr {err:.3e}")
    assert err <= 5e-3


@pytest.mark.parametrize("prec", [dd.F32, dd.F16])
def test_two_level_solve(prec):
    s = Setup(DIMS, BLOCK, eps=0.25, n_stout=2, c_sw=1.7, m0=-0.07, prec=prec, seed=92)
    b = synth.gaussian_spinor(s.V, 905)
    tv = np.stack([synth.gaussian_spinor(s.V, 950 + k) for k in range(12)])
    mg = dd.Multigrid(s.op, tv, setup_iters=3, coarse_max_iter=24, coarse_tol=0.05, sweeps=4, mr_steps=4)
    x, info = s.op.solve(b, tol=1e-10, mg=mg)
    assert info[0]["status"] == 0
    assert relerr(s.ref.apply(x), b) <= 1e-10
    _, info_sap = s.op.solve(b, tol=1e-10)
    assert info[0]["iterations"] < info_sap[0]["iterations"], (info[0]["iterations"], info_sap[0]["iterations"])
    mg.close()
    s.close()


def test_two_level_batched_equals_single():
    """Several right-hand sides in one batched two-level solve (one coarse
    workspace per slot) give the same iterates as each solved alone."""
    s = Setup(DIMS, BLOCK, eps=0.25, n_stout=2, c_sw=1.7, m0=-0.07, prec=dd.F32, seed=93)
    tv = np.stack([synth.gaussian_spinor(s.V, 970 + k) for k in range(8)])
    mg = dd.Multigrid(s.op, tv, setup_iters=3, coarse_max_iter=16, coarse_tol=0.05, sweeps=3, mr_steps=4)
    bs = np.stack([synth.gaussian_spinor(s.V, 980 + r) for r in range(3)])
    xb, infob = s.op.solve(bs, tol=1e-10, mg=mg)
    for r in range(3):
        x1, info1 = s.op.solve(bs[r], tol=1e-10, mg=mg)
        assert np.array_equal(x1, xb[r])
        assert info1[0]["iterations"] == infob[r]["iterations"]
        assert relerr(s.ref.apply(xb[r]), bs[r]) <= 1e-10
    mg.close()
    s.close()


def test_two_level_through_server():
    """Requests that carry a two-level preconditioner, served next to plain
    SAP requests on the same operator, match their solo solves."""
    s = Setup(DIMS, BLOCK, eps=0.25, n_stout=2, c_sw=1.7, m0=-0.07, prec=dd.F32, seed=94)
    tv = np.stack([synth.gaussian_spinor(s.V, 990 + k) for k in range(8)])
    mg = dd.Multigrid(s.op, tv, setup_iters=3, coarse_max_iter=16, coarse_tol=0.05, sweeps=3, mr_steps=4)
    srv = dd.Server(max_slots=4, max_batch_rhs=4)
    jobs = []
    for k in range(4):
        b = synth.gaussian_spinor(s.V, 995 + k)
        use = mg if k % 2 == 0 else None
        jobs.append((b, use, srv.submit(s.op, b, tol=1e-10, mg=use)))
    for b, use, t in jobs:
        st, x, info = srv.wait(t)
        assert st == dd.DONE
        x1, _ = s.op.solve(b, tol=1e-10, mg=use)
        assert np.array_equal(x, x1.reshape(x.shape))
        assert relerr(s.ref.apply(x), b) <= 1e-10
    srv.close()
    mg.close()
    s.close()


def test_two_level_refuses_512_site_aggregates():
    """Aggregates are the Schwarz blocks and the set-up kernels take one
    thread per site of a block, at most 256: an operator on 8 x 4^3 blocks is
    refused with DD_EINVAL and a message naming the limit."""
    s = Setup((16, 8, 8, 8), (8, 4, 4, 4), prec=dd.F32, seed=71)
    tv = np.stack([synth.gaussian_spinor(s.V, 72 + k) for k in range(4)])
    with pytest.raises(dd.DDError) as e:
        dd.Multigrid(s.op, tv, setup_iters=0, coarse_max_iter=8)
    assert e.value.code == -1 and "256" in str(e.value)
    s.close()


def test_two_level_refuses_f16n_operators():
    """The two-level set-up has no DD_F16N path: such an operator is refused
    with DD_EINVAL before any work."""
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), prec=dd.F16N, seed=73)
    tv = np.stack([synth.gaussian_spinor(s.V, 74 + k) for k in range(4)])
    with pytest.raises(dd.DDError) as e:
        dd.Multigrid(s.op, tv, setup_iters=0, coarse_max_iter=8)
    assert e.value.code == -1 and "F16N" in str(e.value)
    s.close()
