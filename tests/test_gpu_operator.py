"""GPU parity of the operator set-up and of apply_D against the FP64 oracle.

Tolerances (relative L2 over the whole result): FP64 1e-13; FP32 1e-6 and
FP16 1e-3 (the Dslash bounds the specification states); BF16 1e-2, derived
from its unit roundoff 2^-8 = 3.9e-3 on inputs, links and clover; F16N (FP16
operator tiles, spinors in 16-bit fixed point with a per-site scale) 1e-3,
as FP16: its tiles round as FP16's, its spinors to 2^-16 of the site's
largest component, well inside that bound. Inputs are
rounded to the storage precision by the library, the oracle gets the exact
FP64 values, so the bound covers storage rounding end to end.
"""
import numpy as np
import pytest

import oracle
import paper_1710_07041_gb300 as dd
import synth
from gpu_common import Setup, relerr

pytestmark = pytest.mark.gpu

TOL = {dd.F64: 1e-13, dd.F32: 1e-6, dd.F16: 1e-3, dd.BF16: 1e-2, dd.F16N: 1e-3}
SHAPES = [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 4, 12), (2, 2, 2, 2)), ((8, 8, 8, 8), (4, 4, 4, 4)),
          ((16, 8, 8, 8), (4, 4, 2, 4)), ((16, 8, 8, 8), (8, 4, 4, 4))]


@pytest.mark.parametrize("dims,block", SHAPES)
def test_clover_blocks_match_oracle(dims, block):
    s = Setup(dims, block, eps=0.4, n_stout=1, c_sw=1.7, m0=-0.05, prec=dd.F64, seed=5)
    A = s.op.clover()
    ref = s.ref.A
    for h in range(2):
        want = ref[:, 6 * h:6 * h + 6, 6 * h:6 * h + 6]
        assert abs(A[:, h] - want).max() < 1e-13
    s.close()


@pytest.mark.parametrize("prec", [dd.F64, dd.F32, dd.F16, dd.BF16, dd.F16N])
@pytest.mark.parametrize("dims,block", SHAPES)
def test_apply_D_matches_oracle(prec, dims, block):
    s = Setup(dims, block, eps=0.3, n_stout=1, c_sw=1.7, m0=-0.02, prec=prec, seed=7)
    psi = synth.gaussian_spinor(s.V, 8)
    fin = s.lat.to_field(psi, prec)
    fout = s.lat.new_field(prec)
    s.op.apply_D(prec, fin, fout)
    got = s.lat.from_field(fout, prec)
    want = s.ref.apply(psi)
    assert relerr(got, want) <= TOL[prec]
    s.close()


@pytest.mark.parametrize("prec", [dd.F64, dd.F32, dd.F16])
def test_apply_D_batched_equals_single(prec):
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), prec=prec, seed=9)
    psi = np.stack([synth.gaussian_spinor(s.V, 20 + r) for r in range(3)])
    fin = s.lat.to_field(psi, prec)
    fout = s.lat.new_field(prec, 3)
    s.op.apply_D(prec, fin, fout, nrhs=3)
    batched = s.lat.from_field(fout, prec, 3)
    for r in range(3):
        f1 = s.lat.to_field(psi[r], prec)
        o1 = s.lat.new_field(prec)
        s.op.apply_D(prec, f1, o1)
        assert np.array_equal(s.lat.from_field(o1, prec), batched[r])
    s.close()


def test_periodic_time_and_free_field():
    """Free field with periodic time: D is diagonal in momentum space."""
    dims = (4, 4, 4, 8)
    U = synth.unit_gauge(dims)
    s = Setup(dims, (2, 2, 2, 2), c_sw=1.0, m0=0.1, prec=dd.F64, U=U, antiperiodic=False)
    psi = synth.gaussian_spinor(s.V, 3)
    f = s.lat.to_field(psi, dd.F64)
    o = s.lat.new_field(dd.F64)
    s.op.apply_D(dd.F64, f, o)
    assert relerr(s.lat.from_field(o, dd.F64), s.ref.apply(psi)) < 1e-14
    s.close()


def _bf16_rne(x):
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


@pytest.mark.parametrize("prec", [dd.F64, dd.F32, dd.F16, dd.BF16])
def test_pack_rounds_to_nearest_even(prec):
    lat = dd.Lattice((4, 4, 4, 4), (2, 2, 2, 2))
    psi = synth.gaussian_spinor(lat.V, 4) * 3.0
    back = lat.from_field(lat.to_field(psi, prec), prec)
    rounders = {dd.F64: lambda v: v, dd.F32: lambda v: v.astype(np.float32).astype(np.float64),
                dd.F16: lambda v: v.astype(np.float16).astype(np.float64), dd.BF16: _bf16_rne}
    r = rounders[prec]
    want = r(psi.real) + 1j * r(psi.imag)
    assert np.array_equal(back, want)
    lat.close()


def _fixed16_site_round(psi):
    """The DD_F16N storage of each site, written out: scale n = FP32 of the
    largest |component| of the site's 24 reals; q = round-half-even(v *
    (32767 / n)) in FP64, |q| <= 32767; the value read back is FP32 q times
    the FP32 product n * (1 / 32767)."""
    v = np.stack([psi.real, psi.imag], axis=-1).reshape(psi.shape[0], 24)
    n = np.abs(v).max(axis=1).astype(np.float32)
    inv = np.where(n > 0, 32767.0 / np.where(n > 0, n.astype(np.float64), 1.0), 0.0)
    q = np.clip(np.rint(v * inv[:, None]), -32767, 32767)
    step = (n * (np.float32(1.0) / np.float32(32767.0))).astype(np.float32)
    back = (q.astype(np.float32) * step[:, None]).astype(np.float64).reshape(psi.shape[0], 12, 2)
    return (back[..., 0] + 1j * back[..., 1]).reshape(psi.shape)


def test_pack_f16n_matches_its_definition():
    """F16N pack and unpack, bit for bit against the definition above, on
    sites of very different magnitudes (the per-site scale follows them) and
    an all-zero site."""
    lat = dd.Lattice((4, 4, 4, 4), (2, 2, 2, 2))
    psi = synth.gaussian_spinor(lat.V, 6)
    psi *= (10.0 ** np.linspace(-12, 6, lat.V))[:, None, None]
    psi[5] = 0
    back = lat.from_field(lat.to_field(psi, dd.F16N), dd.F16N)
    assert np.array_equal(back, _fixed16_site_round(psi))
    # 2^-16 of the site's largest component at most
    err = np.abs(back - psi).reshape(lat.V, -1).max(axis=1)
    big = np.abs(psi).reshape(lat.V, -1).max(axis=1)
    assert np.all(err <= big * 2.0 ** -15)
    lat.close()


def test_fp16_rounding_golden():
    """Ties and near-ties of FP32/FP64 -> FP16 rounding (round-to-nearest-even,
    the mode of the paper's half-precision store, Sec. 3.1 Listing 1)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fp16_rne.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    lat = dd.Lattice((4, 4, 4, 4), (2, 2, 2, 2))
    psi = np.zeros((lat.V, 4, 3), dtype=np.complex128)
    vals = [float.fromhex(a) for a, _ in rows]
    want = [float.fromhex(b) for _, b in rows]
    psi.reshape(-1)[:len(vals)] = vals
    back = lat.from_field(lat.to_field(psi, dd.F16), dd.F16).reshape(-1)[:len(vals)]
    assert np.array_equal(back.real, np.array(want))
    lat.close()


@pytest.mark.parametrize("prec", [dd.F32, dd.F16])
def test_reported_true_residual_matches_oracle(prec):
    """The relative residual a mixed-precision solve reports (FP64 true
    residual on the device) equals the oracle's FP64 recomputation to a few
    digits (rounding of D x is ~1e-16 of |b|, far below a 1e-11 residual)."""
    s = Setup((8, 8, 8, 16), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.02, prec=prec, seed=17)
    b = synth.gaussian_spinor(s.V, 18)
    x, info = s.op.solve(b, tol=1e-10)
    want = relerr(s.ref.apply(x), b)
    assert want <= 1e-10
    assert abs(info[0]["true_rel_residual"] - want) <= 0.02 * want, (info[0]["true_rel_residual"], want)
    s.close()


def test_apply_D_more_rhs_than_one_launch():
    """70 right-hand sides: the library splits them into launches of at most
    64 (the per-launch pointer table); every result equals its single apply."""
    s = Setup((4, 4, 4, 8), (2, 2, 2, 2), prec=dd.F32, seed=10)
    n = 70
    psi = np.stack([synth.gaussian_spinor(s.V, 200 + r) for r in range(n)])
    fin = s.lat.to_field(psi, dd.F32)
    fout = s.lat.new_field(dd.F32, n)
    s.op.apply_D(dd.F32, fin, fout, nrhs=n)
    batched = s.lat.from_field(fout, dd.F32, n)
    for r in (0, 63, 64, 69):
        o1 = s.lat.new_field(dd.F32)
        s.op.apply_D(dd.F32, s.lat.to_field(psi[r], dd.F32), o1)
        assert np.array_equal(s.lat.from_field(o1, dd.F32), batched[r])
    assert relerr(batched[69], s.ref.apply(psi[69])) <= 1e-6
    s.close()


@pytest.mark.parametrize("nrhs", [1, 2])
def test_apply_D_double_float_matches_oracle(nrhs):
    """DD_F64_DF: FP64 fields, double-float arithmetic on the operator's
    pre-split fields (the true-residual operator of mixed-precision solves).
    Each operation errs by a few units of 2^-44 of its operands; an output
    sums ~100 terms of the input's size, so 1e-12 relative L2 leaves margin
    while excluding FP32 arithmetic (~1e-7)."""
    s = Setup((8, 8, 8, 16), (4, 4, 4, 4), eps=0.3, n_stout=1, c_sw=1.7, m0=-0.02, prec=dd.F32, seed=15)
    b = np.stack([synth.gaussian_spinor(s.V, 16 + r) for r in range(nrhs)])
    fin, fout = s.lat.to_field(b, dd.F64), s.lat.new_field(dd.F64, nrhs)
    s.op.apply_D(dd.F64_DF, fin, fout, nrhs=nrhs)
    got = s.lat.from_field(fout, dd.F64, nrhs).reshape(nrhs, s.V, 4, 3)
    for r in range(nrhs):
        assert relerr(got[r], s.ref.apply(b[r])) <= 1e-12
    s.close()
    s64 = Setup((4, 4, 4, 8), (2, 2, 2, 2), prec=dd.F64, seed=3)   # FP64 smoother: no split fields
    f = s64.lat.new_field(dd.F64)
    with pytest.raises(dd.DDError):
        s64.op.apply_D(dd.F64_DF, f, s64.lat.new_field(dd.F64))
    s64.close()


@pytest.mark.parametrize("prec,tol", [(dd.F32, 1e-6), (dd.F16, 2e-3), (dd.BF16, 2e-2)])
def test_links_rebuilt_third_row(prec, tol):
    """The Dslash fields of 32- and 16-bit operators store two rows of each
    SU(3) link and rebuild the third as conj(row0 x row1). A point source
    psi = delta(n + mu) e_{spin 0, colour c} gives, at site n, the spin-0
    entries -1/2 U_mu(n)[a][c] (the forward hop; gamma_mu has no diagonal
    entry in the chiral basis; times -1 across the antiperiodic time edge):
    every column of U_mu(n), including the rebuilt row, against the FP64
    input link."""
    import torch
    dims = (8, 8, 8, 8)
    s = Setup(dims, (4, 4, 4, 4), eps=0.3, n_stout=1, prec=prec, seed=31)
    L = {0: dims[3], 1: dims[2], 2: dims[1], 3: dims[0]}   # extent by direction (x, y, z, t)

    def site(c):   # canonical index of coordinates (x, y, z, t)
        return c[0] + dims[3] * (c[1] + dims[2] * (c[2] + dims[1] * c[3]))

    worst = 0.0
    for n_c in ((1, 2, 3, 4), (3, 0, 5, 7)):
        n = site(n_c)
        for mu in range(4):
            m_c = list(n_c)
            m_c[mu] = (m_c[mu] + 1) % L[mu]
            m = site(m_c)
            for c in range(3):
                psi = np.zeros((s.V, 4, 3), dtype=np.complex128)
                psi[m, 0, c] = 1.0
                fin, fout = s.lat.to_field(psi, prec), s.lat.new_field(prec)
                s.op.apply_D(prec, fin, fout)
                col = -2.0 * s.lat.from_field(fout, prec)[n, 0, :]
                # a hop across the time edge carries the antiperiodic sign
                sign = -1.0 if (mu == 3 and n_c[3] == L[3] - 1) else 1.0
                want = sign * s.U[n, mu, :, c]
                worst = max(worst, float(np.abs(col - want).max()))
    torch.cuda.synchronize()
    assert worst <= tol, worst
    s.close()


def test_non_su3_links_refused():
    """Two-row link storage needs special unitary links: a gauge field with
    one link multiplied by a phase (unitary, determinant != 1) is refused at
    operator creation, for every storage precision."""
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, 0.3, 0, 0.1, seed=5)
    U[17, 2] *= np.exp(0.5j)
    lat = dd.Lattice(dims, (2, 2, 2, 2))
    gauge = dd.Gauge(lat, U)
    for prec in (dd.F64, dd.F32, dd.F16):
        with pytest.raises(dd.DDError) as e:
            dd.Op(gauge, 1.0, 0.1, prec)
        assert e.value.code == -1 and "special unitary" in str(e.value)
    gauge.close()
    lat.close()
