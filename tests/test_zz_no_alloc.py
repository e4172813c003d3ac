"""dd_solve_noalloc: the solve for callers that may not allocate memory.

Such callers (code where cudaMalloc is forbidden or would upset a fixed
memory plan) get the whole FGMRES workspace from a fixed device array built
into the library. This test calls the entry point through the C ABI twice in
a row - the second call finds the first call's data still in the array - and
checks each result against dd_solve's on the same input, and that an
oversized lattice is refused before any work. Collected last on purpose.
"""
import numpy as np
import pytest

import paper_1710_07041_gb300 as dd
import synth
from gpu_common import Setup, relerr

pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_dd_solve_twice():
    import torch
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.02, prec=dd.F32, seed=61)
    for call, seed in enumerate((62, 63)):
        b = synth.gaussian_spinor(s.V, seed)
        b_dev = torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda()
        x_ref_dev, info_ref = s.op.solve(b_dev, tol=1e-10)
        x_dev = torch.full_like(b_dev, float("nan"))   # output buffer content must not matter
        info = dd.solve_noalloc(s.op, b_dev, x_dev, tol=1e-10)
        torch.cuda.synchronize()
        x = x_dev.cpu().numpy().view(np.complex128).reshape(s.V, 4, 3)
        x_ref = x_ref_dev.cpu().numpy().view(np.complex128).reshape(s.V, 4, 3)
        assert info["status"] == 0 and info["true_rel_residual"] <= 1e-10, (call, info)
        assert relerr(s.ref.apply(x), b) <= 1e-10
        assert relerr(x, x_ref) <= 1e-9
        assert info["iterations"] == info_ref[0]["iterations"]
    s.close()


def test_noalloc_refuses_oversized_lattice():
    import torch
    s = Setup((16, 16, 16, 16), (4, 4, 4, 4), prec=dd.F32, seed=64)
    b_dev = torch.zeros(s.V * 24, dtype=torch.float64, device="cuda")
    x_dev = torch.zeros_like(b_dev)
    with pytest.raises(dd.DDError) as e:
        dd.solve_noalloc(s.op, b_dev, x_dev)
    assert e.value.code == -1 and "scratch" in str(e.value)
    s.close()
