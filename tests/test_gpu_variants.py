"""Every launch variant the autotuner can pick, forced one at a time
(DD_TUNE_VARIANT), against the FP64 oracle: the Schwarz smoother's
shared-memory layouts (all tiles staged with one or two CTAs per SM, links
only staged, nothing staged; for 16-bit storage also the two-CTA layouts with
the MR loop unrolled by parity; for 32- and 16-bit storage the links staged
with the clover blocks in tensor memory), each with the one-CTA-per-block and the
persistent grid, and the eight Dslash launch variants (four launch shapes,
each with the clover tiles read through L1 or past it); on the 4^4 block shape
and, in the second half, on the 8 x 4^3 block (512-thread CTAs, the shape
the batched workload picks) in every precision, and FP64 on the 4^4 shape.
Bounds as in test_gpu_sap.py and test_gpu_operator.py."""
import os

import numpy as np
import pytest

import paper_1710_07041_gb300 as dd
import synth
from gpu_common import Setup, relerr

pytestmark = pytest.mark.gpu

SAP_TOL = {dd.F64: 1e-12, dd.F32: 5e-7, dd.F16: 1.5e-3, dd.BF16: 1.2e-2, dd.F16N: 1e-3}
DSLASH_TOL = {dd.F64: 1e-13, dd.F32: 1e-6, dd.F16: 1e-3, dd.BF16: 1e-2, dd.F16N: 1e-3}


class forced_variant:
    def __init__(self, k):
        self.k = k

    def __enter__(self):
        self.old = os.environ.get("DD_TUNE_VARIANT")
        os.environ["DD_TUNE_VARIANT"] = str(self.k)

    def __exit__(self, *a):
        if self.old is None:
            del os.environ["DD_TUNE_VARIANT"]
        else:
            os.environ["DD_TUNE_VARIANT"] = self.old


@pytest.fixture(scope="module", params=[dd.F32, dd.F16, dd.BF16, dd.F16N])
def setup(request):
    s = Setup((8, 8, 8, 16), (4, 4, 4, 4), eps=0.3, n_stout=1, c_sw=1.7, m0=-0.02, prec=request.param, seed=13)
    b = synth.gaussian_spinor(s.V, 14)
    yield s, b, s.ref.sap((4, 4, 4, 4), b, 2, 4), s.ref.apply(b)
    s.close()


@pytest.mark.parametrize("k", range(12))
def test_sap_variant(setup, k):
    s, b, want, _ = setup
    fb = s.lat.to_field(b, s.prec)
    fx = s.lat.new_field(s.prec)
    with forced_variant(k):
        s.op.sap_smooth(fb, fx, 2, 4, x_is_zero=True)
    dd.device_status()   # no staging wait expired
    got = s.lat.from_field(fx, s.prec)
    assert relerr(got, want) <= SAP_TOL[s.prec]


@pytest.mark.parametrize("k", range(8))
def test_dslash_variant(setup, k):
    s, b, _, want = setup
    fin, fout = s.lat.to_field(b, s.prec), s.lat.new_field(s.prec)
    with forced_variant(k):
        s.op.apply_D(s.prec, fin, fout)
    got = s.lat.from_field(fout, s.prec)
    assert relerr(got, want) <= DSLASH_TOL[s.prec]


# The 8 x 4^3 block (SHAPE 2: 512 threads per CTA) in every precision, and
# FP64 on the 4^4 block: the Schwarz layouts (tiles in shared memory; for 32-
# and 16-bit storage also the clover blocks in tensor memory), each with one
# CTA per block and the persistent grid; eight Dslash launch variants.
@pytest.fixture(scope="module",
                params=[(dd.F64, (4, 4, 4, 4)), (dd.F64, (8, 4, 4, 4)), (dd.F32, (8, 4, 4, 4)),
                        (dd.F16, (8, 4, 4, 4)), (dd.BF16, (8, 4, 4, 4))],
                ids=["f64-4^4", "f64-8x4^3", "f32-8x4^3", "f16-8x4^3", "bf16-8x4^3"])
def setup2(request):
    prec, block = request.param
    s = Setup((16, 8, 8, 8), block, eps=0.3, n_stout=1, c_sw=1.7, m0=-0.02, prec=prec, seed=15)
    b = synth.gaussian_spinor(s.V, 16)
    yield s, b, s.ref.sap(block, b, 2, 4), s.ref.apply(b)
    s.close()


@pytest.mark.parametrize("k", range(4))
def test_sap_variant_shapes(setup2, k):
    s, b, want, _ = setup2
    fb = s.lat.to_field(b, s.prec)
    fx = s.lat.new_field(s.prec)
    with forced_variant(k):
        s.op.sap_smooth(fb, fx, 2, 4, x_is_zero=True)
    dd.device_status()
    got = s.lat.from_field(fx, s.prec)
    assert relerr(got, want) <= SAP_TOL[s.prec]


@pytest.mark.parametrize("k", range(8))
def test_dslash_variant_shapes(setup2, k):
    s, b, _, want = setup2
    fin, fout = s.lat.to_field(b, s.prec), s.lat.new_field(s.prec)
    with forced_variant(k):
        s.op.apply_D(s.prec, fin, fout)
    got = s.lat.from_field(fout, s.prec)
    assert relerr(got, want) <= DSLASH_TOL[s.prec]
