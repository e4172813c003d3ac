"""Batched and served solves: every right-hand side gets the same solution
alone and in a mixed batch (bit-identical: its reductions and decisions do
not depend on its batch mates), requests on lattices of different sizes
are served at the same time - in one worker whose Schwarz launches cover
all their lattices - and the server admits by memory budget and cancels."""
import time

import numpy as np
import pytest

import paper_1710_07041_gb300 as dd
import synth
from gpu_common import Setup, relerr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [dd.F32, dd.F16, dd.F16N])
def test_batched_solve_equals_single(prec):
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.02, prec=prec, seed=31)
    bs = np.stack([synth.gaussian_spinor(s.V, 40 + r) for r in range(3)])
    xb, infob = s.op.solve(bs, tol=1e-10)
    for r in range(3):
        x1, info1 = s.op.solve(bs[r], tol=1e-10)
        assert np.array_equal(x1, xb[r])
        assert info1[0]["iterations"] == infob[r]["iterations"]
        assert relerr(s.ref.apply(xb[r]), bs[r]) <= 1e-10
    s.close()


def test_server_mixed_lattices_match_solo():
    small = Setup((8, 8, 8, 8), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=0.01, prec=dd.F32, seed=41)
    large = Setup((16, 8, 8, 8), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.01, prec=dd.F16, seed=42)
    srv = dd.Server(max_slots=4, max_batch_rhs=4)
    jobs = []
    for k in range(6):
        s = small if k % 2 == 0 else large
        nrhs = 1 + k % 3
        b = np.stack([synth.gaussian_spinor(s.V, 100 + 10 * k + r) for r in range(nrhs)])
        jobs.append((s, b, srv.submit(s.op, b if nrhs > 1 else b[0], tol=1e-10)))
        time.sleep(0.01)
    for s, b, t in jobs:
        st, x, info = srv.wait(t)
        assert st == dd.DONE, info
        x = x.reshape(b.shape)
        for r in range(b.shape[0]):
            assert relerr(s.ref.apply(x[r]), b[r]) <= 1e-10
            x1, _ = s.op.solve(b[r], tol=1e-10)
            assert np.array_equal(x1, x[r])
    st = srv.stats()
    assert st["completed"] == 6 and st["failed"] == 0 and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()
    small.close()
    large.close()


def test_server_serves_f16n_operators():
    """Requests on an operator with DD_F16N smoother storage: served to 1e-10
    and bitwise the same as the solo solves."""
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.02, prec=dd.F16N, seed=47)
    srv = dd.Server(max_slots=4, max_batch_rhs=4)
    bs = [np.stack([synth.gaussian_spinor(s.V, 150 + 10 * k + r) for r in range(1 + k)]) for k in range(2)]
    tickets = [srv.submit(s.op, b if b.shape[0] > 1 else b[0], tol=1e-10) for b in bs]
    for b, t in zip(bs, tickets):
        st, x, info = srv.wait(t)
        assert st == dd.DONE, info
        x = x.reshape(b.shape)
        for r in range(b.shape[0]):
            assert relerr(s.ref.apply(x[r]), b[r]) <= 1e-10
            x1, _ = s.op.solve(b[r], tol=1e-10)
            assert np.array_equal(x1, x[r])
    srv.close()
    s.close()


def test_server_budget_and_cancel():
    s = Setup((8, 8, 8, 8), (4, 4, 4, 4), prec=dd.F32, seed=43)
    b = synth.gaussian_spinor(s.V, 44)
    tiny = dd.Server(hbm_budget_bytes=1 << 20, max_slots=2, max_batch_rhs=2)
    with pytest.raises(dd.DDError) as e:
        tiny.submit(s.op, b)
    assert e.value.code == -7   # DD_EBUSY
    tiny.close()
    srv = dd.Server(max_slots=1, max_batch_rhs=1)
    t1 = srv.submit(s.op, b, tol=1e-14, max_iter=100000)   # long-running
    t2 = srv.submit(s.op, b)
    srv.cancel(t1)
    st1, _, _ = srv.wait(t1)
    st2, x2, _ = srv.wait(t2)
    assert st1 == dd.CANCELLED and st2 == dd.DONE
    assert relerr(s.ref.apply(x2), b) <= 1e-10
    assert dd.lib().dd_cancel(srv.handle, 999999) == -8   # DD_ENOTFOUND
    srv.close()
    s.close()


def test_server_lattices_share_one_worker_and_overlap():
    """Requests on three lattices of different sizes (same smoother
    precision and block shape) are served by one worker: their right-hand
    sides sit in its slots together, each Arnoldi step smoothing all of them
    in one launch per colour phase. The polling below sees the requests
    RUNNING at overlapping times; every result is bit for bit the solo
    solve's and reaches 1e-10 by the oracle's operator."""
    sizes = [((8, 8, 8, 8), 61), ((8, 8, 8, 16), 62), ((16, 8, 8, 8), 63)]
    setups = [Setup(d, (4, 4, 4, 4), eps=0.25, n_stout=2, c_sw=1.7, m0=-0.01, prec=dd.F16, seed=sd)
              for d, sd in sizes]
    srv = dd.Server(max_slots=8, max_batch_rhs=8)
    jobs = []
    for k, s in enumerate(setups):
        b = np.stack([synth.gaussian_spinor(s.V, 200 + 10 * k + r) for r in range(2)])
        jobs.append((s, b, srv.submit(s.op, b, tol=1e-10)))
    running = {t: None for _, _, t in jobs}
    done, xs = {}, {t: np.zeros(b.shape, dtype=np.complex128) for _, b, t in jobs}
    t0 = time.perf_counter()
    state = dd.ctypes.c_int()
    while len(done) < len(jobs) and time.perf_counter() - t0 < 600:
        now = time.perf_counter() - t0
        for s, b, t in jobs:
            if t in done:
                continue
            # x is written (and the ticket released) once the request is done
            assert dd.lib().dd_poll(srv.handle, t, dd.ctypes.byref(state), dd._ptr(xs[t]), None) == 0
            if state.value == dd.RUNNING and running[t] is None:
                running[t] = now
            if state.value in (dd.DONE, dd.FAILED, dd.CANCELLED):
                done[t] = (state.value, now)
        time.sleep(0.0005)
    assert len(done) == len(jobs) and all(v[0] == dd.DONE for v in done.values()), done
    ivals = [(running[t] if running[t] is not None else done[t][1], done[t][1]) for _, _, t in jobs]
    overlaps = sum(1 for i in range(len(ivals)) for j in range(i + 1, len(ivals))
                   if max(ivals[i][0], ivals[j][0]) < min(ivals[i][1], ivals[j][1]))
    assert overlaps >= 1, ivals
    srv.close()
    for s, b, t in jobs:
        for r in range(2):
            assert relerr(s.ref.apply(xs[t][r]), b[r]) <= 1e-10
            x1, _ = s.op.solve(b[r], tol=1e-10)
            assert np.array_equal(x1, xs[t][r])
    for s in setups:
        s.close()
