"""The index-checking build (build.py --checked, -DDD_CHECKED): every main
global and shared-memory access path checks its index and counts (and
clamps) any out-of-range one, in place of a memory checker. The test builds
that variant, runs Dslash, Schwarz, solve and two-level parity cases through
it in a child process (DD_LIBRARY selects the build) and requires both parity
with the oracle and a zero count (dd_device_status)."""
import os
import subprocess
import sys

import pytest

import paper_1710_07041_gb300 as dd

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
import paper_1710_07041_gb300 as dd
import synth
from gpu_common import Setup, relerr
from oracle.twolevel import TwoLevel

for dims, block in (((8, 8, 8, 8), (4, 4, 4, 4)), ((4, 4, 8, 8), (2, 2, 2, 2)), ((16, 8, 8, 8), (8, 4, 4, 4))):
    for prec, tol_d, tol_s in ((dd.F32, 1e-6, 1e-5), (dd.F16, 1e-3, 1e-2)):
        s = Setup(dims, block, eps=0.3, n_stout=1, c_sw=1.7, m0=-0.02, prec=prec, seed=71)
        b = synth.gaussian_spinor(s.V, 72)
        fin, fout = s.lat.to_field(b, prec), s.lat.new_field(prec)
        s.op.apply_D(prec, fin, fout)
        assert relerr(s.lat.from_field(fout, prec), s.ref.apply(b)) <= tol_d, (dims, prec)
        fx = s.lat.new_field(prec)
        s.op.sap_smooth(fin, fx, 2, 3)
        assert relerr(s.lat.from_field(fx, prec), s.ref.sap(block, b, 2, 3)) <= tol_s, (dims, prec)
        x, info = s.op.solve(b, tol=1e-10)
        assert relerr(s.ref.apply(x), b) <= 1e-10
        s.close()
s = Setup((8, 8, 8, 8), (4, 4, 4, 4), eps=0.3, n_stout=1, c_sw=1.0, m0=-0.05, prec=dd.F32, seed=91)
tv = np.stack([synth.gaussian_spinor(s.V, 900 + k) for k in range(6)])
mg = dd.Multigrid(s.op, tv, setup_iters=0, coarse_max_iter=12, coarse_tol=0.0, sweeps=2, mr_steps=3)
tl = TwoLevel(s.ref, (4, 4, 4, 4), tv)
r = synth.gaussian_spinor(s.V, 904)
rf, xf = s.lat.to_field(r, dd.F32), s.lat.new_field(dd.F32)
mg.precondition(rf, xf)
want = tl.precondition(s.lat.from_field(rf, dd.F32), (4, 4, 4, 4), sweeps=2, nmr=3, coarse_restart=12,
                       coarse_iter=12, coarse_tol=0.0)
assert relerr(s.lat.from_field(xf, dd.F32), want) <= 5e-3
mg.close()
s.close()
dd.device_status()   # raises if the checked build caught an out-of-range index
print("checked build: parity and no out-of-range index")
'''


def test_checked_build_parity_and_no_out_of_range_index():
    path = dd._build.build(checked=True)
    env = dict(os.environ, DD_LIBRARY=path,
               PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests"), os.environ.get("PYTHONPATH", "")]))
    p = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    assert "no out-of-range index" in p.stdout
