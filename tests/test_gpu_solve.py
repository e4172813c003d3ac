"""SAP-preconditioned FGMRES on the GPU: every solve reaches a true relative
residual of 1e-10, measured by the FP64 oracle's own operator on the GPU's
solution, and agrees with the oracle's FGMRES / dense LU solution."""
import numpy as np
import pytest

import paper_1710_07041_gb300 as dd
import synth
from gpu_common import Setup, relerr

pytestmark = pytest.mark.gpu


def true_res(s, x, b):
    return relerr(s.ref.apply(x), b)


def test_plain_fp64_workload_4x4x4x4_matches_lu():
    """exp(i 0.3 H) links, c_sw = 1, m0 = 0.1, 2^4 blocks, 4 sweeps, 3 MR,
    FGMRES(16) to 1e-10; checked against a dense LU solve of D."""
    s = Setup((4, 4, 4, 4), (2, 2, 2, 2), eps=0.3, n_stout=0, c_sw=1.0, m0=0.1, prec=dd.F64, seed=1)
    b = synth.gaussian_spinor(s.V, 2)
    x, info = s.op.solve(b, tol=1e-10, restart=16, sweeps=4, mr_steps=3)
    assert info[0]["status"] == 0
    assert true_res(s, x, b) <= 1e-10
    D = s.ref.dense()
    x_lu = np.linalg.solve(D, b.reshape(-1))
    kappa = np.linalg.cond(D)
    assert relerr(x.reshape(-1), x_lu) <= kappa * 1e-10
    xo, ok, st = s.ref.fgmres(s.block, b, 16, 1e-10, 500, 4, 3)
    assert ok and info[0]["iterations"] <= st["iterations"] + 2
    s.close()


@pytest.mark.parametrize("prec", [dd.F64, dd.F32, dd.F16, dd.BF16, dd.F16N])
def test_mixed_precision_solve_reaches_1e10(prec):
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.02, prec=prec, seed=21)
    b = synth.gaussian_spinor(s.V, 22)
    x, info = s.op.solve(b, tol=1e-10, restart=16, sweeps=4, mr_steps=4)
    assert info[0]["status"] == 0, info
    assert true_res(s, x, b) <= 1e-10
    assert info[0]["true_rel_residual"] <= 1e-10
    s.close()


def test_solve_device_buffers_and_initial_guess():
    import torch
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), prec=dd.F32, seed=23)
    b = np.stack([synth.gaussian_spinor(s.V, 24), synth.gaussian_spinor(s.V, 25)])
    bd = torch.from_numpy(b.view(np.float64).copy()).cuda()
    xd, info = s.op.solve(bd, tol=1e-10)
    x = xd.cpu().numpy().view(np.complex128).reshape(2, s.V, 4, 3)
    for r in range(2):
        assert true_res(s, x[r], b[r]) <= 1e-10
    # restarting from the solution converges immediately
    x2, info2 = s.op.solve(b[0], x=x[0].copy(), use_x0=True, tol=1e-10)
    assert info2[0]["iterations"] == 0
    s.close()


def test_not_converged_and_zero_rhs():
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), prec=dd.F32, seed=26)
    b = synth.gaussian_spinor(s.V, 27)
    x, info = s.op.solve(b, tol=1e-14, max_iter=3, raise_on_notconv=False)
    assert info[0]["status"] == -4 and info[0]["iterations"] == 3
    with pytest.raises(dd.DDError):
        s.op.solve(b, tol=1e-14, max_iter=3)
    x, info = s.op.solve(np.zeros_like(b))
    assert info[0]["status"] == 0 and not x.any()
    s.close()


def test_workspace_cache_reuse_and_release():
    """A solve reuses the workspace the previous one left in the cache (its
    buffers still hold that solve's data): the result is bitwise the same as
    the first solve's. dd_release_workspace gives the memory back."""
    import torch
    s = Setup((8, 8, 8, 16), (4, 4, 4, 4), prec=dd.F32, seed=27)
    b = synth.gaussian_spinor(s.V, 28)
    b2 = synth.gaussian_spinor(s.V, 29)
    dd.release_workspace()
    x1, info1 = s.op.solve(b, tol=1e-10)
    s.op.solve(b2, tol=1e-10)            # leaves different data in the cached buffers
    x3, info3 = s.op.solve(b, tol=1e-10)
    assert info1[0]["status"] == 0 and info3[0]["status"] == 0
    assert info3[0]["iterations"] == info1[0]["iterations"]
    assert np.array_equal(x1, x3)
    assert true_res(s, x3, b) <= 1e-10
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    dd.release_workspace()
    free1 = torch.cuda.mem_get_info()[0]
    # the cached slot: (m + 1) double-float basis fields, m FP32 fields, and
    # scratch - at least the basis, 17 x 24 x 8 bytes per site
    assert free1 - free0 >= 17 * 24 * 8 * s.V
    s.close()


@pytest.mark.parametrize("prec", [dd.F32, dd.F16])
def test_outer_f64_solve_reaches_1e10(prec):
    """The mixed-precision smoother with an IEEE FP64 Krylov basis and FP64
    true residual (outer_f64) converges like the double-float default: same
    target, iteration count within one or two steps."""
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.02, prec=prec, seed=21)
    b = synth.gaussian_spinor(s.V, 22)
    x, info = s.op.solve(b, tol=1e-10, outer_f64=True)
    assert info[0]["status"] == 0, info
    assert true_res(s, x, b) <= 1e-10
    _, info_df = s.op.solve(b, tol=1e-10)
    assert abs(info[0]["iterations"] - info_df[0]["iterations"]) <= 2
    with pytest.raises(dd.DDError):   # not with the two-level preconditioner (its argument check)
        p = dd.SolveParams(1e-10, 16, 100, dd.SapParams(4, 4, 1, 0), 1e-5, dd.HOST, 0, 1, 1)
        dd._check(dd.lib().dd_solve(s.op.handle, dd.ctypes.byref(p), dd._ptr(b), dd._ptr(np.zeros_like(b)), 1,
                                    None, None), "dd_solve")
    s.close()
