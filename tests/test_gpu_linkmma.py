"""The tensor-core measurement of the multi-right-hand-side link product
(dd_bench_link_product): the warp-level MMA form (two site-directions packed
block-diagonally into one m16n8k16 operand, FP16 inputs, FP32 accumulation)
and the FP16-operand CUDA-core form compute the same 6x6 by 6x24 real
products as the FP32 CUDA-core form. Inputs are multiples of 1/64, exact in
FP16, and every product and sum of six is exact in FP32, so the three must
agree to FP32 rounding (here exactly)."""
import pytest

import paper_1710_07041_gb300 as dd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", [0, 1, 2])
def test_link_product_methods_agree(method):
    ms, products, diff = dd.bench_link_product(method, ctas=304, reps=20)
    assert ms > 0 and products == 304 * 64
    assert diff <= 1e-6, diff
