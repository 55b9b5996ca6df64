"""Continuous batching (hm_batch_* and the Python Server) on the GPU.

The bar: a request's solution, iteration count and residual are bitwise the same whether it
runs alone (solve() on that one column) or joins a running batch at any step, next to any
other requests, on one geometry or with a second geometry sharing the GPU.  solve() itself
is checked against the oracle in test_gpu_parity.py.
"""
import numpy as np
import pytest

import paper_2111_13483_gb300 as hm
from paper_2111_13483_gb300 import serve

pytestmark = pytest.mark.gpu


def _rhs(P, count, seed):
    return [V for _, _, V in serve.monostatic_requests(P, count, seed, phi_step_deg=17.0)]


@pytest.fixture(scope="module")
def sphere_mixed(sphere1920):
    h = hm.hmat_create(sphere1920, ordering=1, fill_tol=1e-2, precision=1)
    hm.precond_setup(h)
    return sphere1920, h


@pytest.fixture(scope="module")
def sphere_fp64(sphere1920):
    h = hm.hmat_create(sphere1920, ordering=1, fill_tol=0.0, precision=0)
    hm.precond_setup(h)
    return sphere1920, h


@pytest.fixture(scope="module")
def small_mixed(sphere480):
    h = hm.hmat_create(sphere480, ordering=1, fill_tol=1e-2, precision=1)
    hm.precond_setup(h)
    return sphere480, h


def _alone(h, Vs, tol, restart=30):
    out = []
    for V in Vs:
        I, it, rr, code = hm.solve(h, V, tol=tol, restart=restart)
        out.append((I, int(it[0]), float(rr[0]), code))
    return out


@pytest.mark.parametrize("which", ["sphere_mixed", "sphere_fp64"])
def test_batch_staggered_joins_equal_solve_alone(which, request):
    """Requests join a running 4-slot engine at different steps (more requests than slots,
    so finished slots are reused); each equals its solo solve bitwise."""
    P, h = request.getfixturevalue(which)
    Vs = _rhs(P, 7, seed=11)
    tol = 1e-5
    ref = _alone(h, Vs, tol)
    b = hm.Batch(h, 4, 30)
    try:
        slot_of, res, nxt, step = {}, {}, 0, 0
        while len(res) < len(Vs):
            # admit one request every third step while a slot is free
            if nxt < len(Vs) and step % 3 == 0:
                s = b.submit(Vs[nxt], tol=tol)
                if s is not None:
                    slot_of[s] = nxt
                    nxt += 1
            for s in b.step():
                I, it, rr, code = b.result(s)
                res[slot_of.pop(s)] = (I, it, rr, code)
            step += 1
            assert step < 20000
    finally:
        b.close()
    for i, (I, it, rr, code) in res.items():
        Ia, ita, rra, codea = ref[i]
        assert code == codea == 0
        assert it == ita and rr == rra, i
        assert np.array_equal(I, Ia), i


def test_batch_busy_state_and_single_open(small_mixed):
    P, h = small_mixed
    Vs = _rhs(P, 3, seed=5)
    b = hm.Batch(h, 2, 30)
    try:
        assert b.submit(Vs[0]) is not None and b.submit(Vs[1]) is not None
        assert b.submit(Vs[2]) is None                      # HM_EBUSY: both slots taken
        with pytest.raises(hm.HMError):
            b.result(0)                                     # not finished yet: HM_ESTATE
        with pytest.raises(hm.HMError):
            hm.Batch(h, 2, 30)                              # one batch per handle
        done = []
        for _ in range(5000):
            done += b.step()
            if len(done) == 2:
                break
        assert sorted(done) == [0, 1]
        for s in done:
            I, it, rr, code = b.result(s)
            assert code == 0 and rr <= 1e-4
    finally:
        b.close()
    b2 = hm.Batch(h, 1, 30)                                 # the handle is free again
    b2.close()


def test_batch_device_rhs_and_result(small_mixed):
    torch = pytest.importorskip("torch")
    P, h = small_mixed
    V = _rhs(P, 1, seed=9)[0]
    I0, it0, rr0, _ = hm.solve(h, V, tol=1e-5)
    b = hm.Batch(h, 1, 30)
    try:
        dV = torch.from_numpy(V.copy()).cuda()
        s = b.submit(dV, tol=1e-5)
        fin = []
        while not fin:
            fin = b.step()
        dI = torch.zeros_like(dV)
        _, it, rr, code = b.result(s, out=dI)
        assert code == 0 and it == it0[0]
        assert np.array_equal(dI.cpu().numpy(), I0)
    finally:
        b.close()


def test_server_two_geometries_poisson_mix_equals_alone(sphere_mixed, small_mixed):
    """Two resident geometries, Poisson arrivals faster than service (requests queue and join
    running batches): every result equals its solo solve bitwise, latencies are recorded."""
    (P1, h1), (P2, h2) = sphere_mixed, small_mixed
    R1, R2 = _rhs(P1, 10, seed=21), _rhs(P2, 10, seed=22)
    tol = 1e-4
    ref1, ref2 = _alone(h1, R1, tol), _alone(h2, R2, tol)
    srv = serve.Server({"sphere": h1, "small": h2}, max_slots=4, tol=tol)
    try:
        reqs = serve.run_stream(srv, [("sphere", serve.poisson_arrivals(10, 40.0, 1), R1),
                                      ("small", serve.poisson_arrivals(10, 40.0, 2), R2)])
    finally:
        srv.close()
    by = {"sphere": iter(ref1), "small": iter(ref2)}
    # run_stream returns requests in arrival order; regroup per geometry in submission order
    per = {"sphere": [r for r in reqs if r.geom == "sphere"], "small": [r for r in reqs if r.geom == "small"]}
    for name, rs in per.items():
        for r, V in zip(rs, R1 if name == "sphere" else R2):
            assert np.array_equal(r.V, V)
            Ia, ita, rra, codea = next(by[name])
            assert r.status == codea == 0
            assert r.iters == ita and r.relres == rra
            assert np.array_equal(r.I, Ia)
            assert r.latency > 0 and r.queue_time >= 0
    s = serve.latency_summary(reqs)
    assert s["requests"] == 20 and s["p99_s"] >= s["p50_s"] > 0


def test_server_hbm_budget_limits_slots(small_mixed):
    P, h = small_mixed
    per = hm.Batch.bytes(h, 2, 30) - hm.Batch.bytes(h, 1, 30)
    base = hm.Batch.bytes(h, 1, 30) - per
    srv = serve.Server({"small": h}, hbm_budget=base + 3 * per + per // 2, max_slots=64)
    try:
        assert srv.slots("small") == 3
        Vs = _rhs(P, 5, seed=3)
        reqs = [srv.submit("small", V) for V in Vs]
        for r in reqs:
            r.wait(timeout=300)
            assert r.status == 0
    finally:
        srv.close()
    with pytest.raises(MemoryError):
        serve.Server({"small": h}, hbm_budget=base + per // 2)
