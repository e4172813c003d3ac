"""The kernels' bounded wait for staged data (the Schwarz kernel's bulk-copy
barrier), exercised without a fault: a copy that completes, then a barrier
that is told to expect bytes nobody copies. The wait must expire after about
a second, raise the flag dd_device_status reports (once), and leave the
context usable."""
import time

import numpy as np
import pytest

import paper_1710_07041_gb300 as dd
import synth
from gpu_common import Setup, relerr

pytestmark = pytest.mark.gpu


def test_wait_completes_then_expires():
    dd.device_status()                 # clear anything earlier
    dd.selftest_wait(False)
    dd.device_status()                 # nothing expired
    t0 = time.perf_counter()
    dd.selftest_wait(True)             # DD_OK: the expiry was observed
    waited = time.perf_counter() - t0
    assert 0.2 < waited < 30, waited
    with pytest.raises(dd.DDError):
        dd.device_status()             # the flag is reported once
    dd.device_status()                 # and cleared
    # the context is still usable: a Dslash against the oracle
    s = Setup((4, 4, 4, 8), (2, 2, 2, 2), prec=dd.F32, seed=3)
    b = synth.gaussian_spinor(s.V, 4)
    fin, fout = s.lat.to_field(b, dd.F32), s.lat.new_field(dd.F32)
    s.op.apply_D(dd.F32, fin, fout)
    assert relerr(s.lat.from_field(fout, dd.F32), s.ref.apply(b)) <= 1e-6
    s.close()
