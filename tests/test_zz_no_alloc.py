"""dd_solve_noalloc: the solve for callers that may not allocate memory.

Such callers (code where cudaMalloc is forbidden or would upset a fixed
memory plan) get the whole FGMRES workspace from a fixed device array built
into the library. These tests call the entry point through the C ABI twice
in a row - the second call finds the first call's data still in the array -
and check each result against dd_solve's on the same input and against the
oracle's residual: on the legacy stream, and on a stream of the caller's own
(where ordinary smoother calls would capture and replay CUDA graphs) for an
FP64, an FP32 and an FP16 smoother. A fresh process checks that the call
does no launch-configuration tuning of its own (its first call launches as
many kernels as its second), and an oversized lattice is refused before any
work. Collected last on purpose.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import paper_1710_07041_gb300 as dd
import synth
from gpu_common import Setup, relerr

pytestmark = pytest.mark.gpu


def _to_dev(b):
    import torch
    return torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda()


def _spinor(t, V):
    return t.cpu().numpy().view(np.complex128).reshape(V, 4, 3)


def test_noalloc_solve_matches_dd_solve_twice():
    import torch
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.02, prec=dd.F32, seed=61)
    for call, seed in enumerate((62, 63)):
        b = synth.gaussian_spinor(s.V, seed)
        b_dev = _to_dev(b)
        x_ref_dev, info_ref = s.op.solve(b_dev, tol=1e-10)
        x_dev = torch.full_like(b_dev, float("nan"))   # output buffer content must not matter
        info = dd.solve_noalloc(s.op, b_dev, x_dev, tol=1e-10)
        torch.cuda.synchronize()
        x, x_ref = _spinor(x_dev, s.V), _spinor(x_ref_dev, s.V)
        assert info["status"] == 0 and info["true_rel_residual"] <= 1e-10, (call, info)
        assert relerr(s.ref.apply(x), b) <= 1e-10
        assert relerr(x, x_ref) <= 1e-9
        assert info["iterations"] == info_ref[0]["iterations"]
    s.close()


@pytest.mark.parametrize("prec", [dd.F64, dd.F32, dd.F16, dd.F16N], ids=["f64", "f32", "f16", "f16n"])
def test_noalloc_on_own_stream_twice(prec):
    """On a non-default stream: two calls in a row, each against dd_solve and
    the oracle's residual (FP64 smoother: native FP64 basis; FP16: the
    smoother's output converted into the FP32 preconditioned vectors)."""
    import torch
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.02, prec=prec, seed=65)
    side = torch.cuda.Stream()
    for call, seed in enumerate((66, 67)):
        b = synth.gaussian_spinor(s.V, seed)
        b_dev = _to_dev(b)
        x_ref_dev, info_ref = s.op.solve(b_dev, tol=1e-10)
        torch.cuda.synchronize()
        x_dev = torch.full_like(b_dev, float("nan"))
        side.wait_stream(torch.cuda.current_stream())
        info = dd.solve_noalloc(s.op, b_dev, x_dev, tol=1e-10, stream=side)
        side.synchronize()
        x, x_ref = _spinor(x_dev, s.V), _spinor(x_ref_dev, s.V)
        assert info["status"] == 0 and info["true_rel_residual"] <= 1e-10, (call, info)
        assert relerr(s.ref.apply(x), b) <= 1e-10
        assert relerr(x, x_ref) <= 1e-9
        assert info["iterations"] == info_ref[0]["iterations"]
    s.close()


def test_noalloc_first_call_does_no_tuning():
    """In a fresh process (no tuner cache), the first call must not run the
    autotuner's trial launches: it launches exactly as many kernels as the
    second, identical call."""
    script = textwrap.dedent("""
        import sys
        sys.path[:0] = [{root!r}, {tests!r}]
        import numpy as np, torch
        import paper_1710_07041_gb300 as dd, synth
        from gpu_common import Setup
        s = Setup((8, 8, 8, 8), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.02, prec=dd.F32, seed=68)
        b = torch.from_numpy(synth.gaussian_spinor(s.V, 69).view(np.float64).reshape(-1).copy()).cuda()
        side = torch.cuda.Stream()
        counts, its = [], []
        for _ in range(2):
            x = torch.zeros_like(b)
            n0 = dd.kernel_launches()
            info = dd.solve_noalloc(s.op, b, x, tol=1e-10, stream=side)
            counts.append(dd.kernel_launches() - n0)
            its.append(info["iterations"])
            assert info["status"] == 0 and info["true_rel_residual"] <= 1e-10, info
        assert counts[0] == counts[1] and its[0] == its[1], (counts, its)
        print("launches per call", counts)
        s.close()
    """).format(root=os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                tests=os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("DD_TUNE_CACHE", "DD_TUNE_VARIANT", "DD_TUNE")}
    p = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout + p.stderr


def test_noalloc_refuses_oversized_lattice():
    import torch
    s = Setup((16, 16, 16, 16), (4, 4, 4, 4), prec=dd.F32, seed=64)
    b_dev = torch.zeros(s.V * 24, dtype=torch.float64, device="cuda")
    x_dev = torch.zeros_like(b_dev)
    with pytest.raises(dd.DDError) as e:
        dd.solve_noalloc(s.op, b_dev, x_dev)
    assert e.value.code == -1 and "scratch" in str(e.value)
    s.close()
