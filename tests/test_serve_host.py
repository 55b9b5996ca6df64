"""Host logic of the serving loop (no GPU): admission, slot limits, HBM-budget sizing, request
generators.  The slot engine is replaced by a fake with the same interface."""
import threading

import numpy as np
import pytest

from paper_2111_13483_gb300 import serve


class FakeBatch:
    """Each request needs int(V[0].real) steps; the result is 2 V."""
    opened = []

    def __init__(self, h, slots, restart):
        self.slots, self.restart = slots, restart
        self.live = {}
        self.max_live = 0
        self.admitted = []
        self.lock = threading.Lock()
        FakeBatch.opened.append(self)

    @staticmethod
    def bytes(h, slots, restart):
        return 5000 + 1000 * slots * (restart + 1)

    def submit(self, V, tol=1e-4, maxit=5000):
        for s in range(self.slots):
            if s not in self.live:
                self.live[s] = [int(V[0].real), V]
                self.admitted.append(int(V[1].real))
                self.max_live = max(self.max_live, len(self.live))
                return s
        return None

    def step(self):
        fin = []
        for s, st in self.live.items():
            st[0] -= 1
            if st[0] <= 0:
                fin.append(s)
        return fin

    def result(self, s):
        steps, V = self.live.pop(s)
        return 2 * V, int(V[0].real), 0.0, 0

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    FakeBatch.opened = []
    monkeypatch.setattr(serve.hmsolve, "Batch", FakeBatch)
    return FakeBatch


class H:
    n = 4


def _req(steps, ident):
    V = np.zeros(4, dtype=np.complex128)
    V[0], V[1] = steps, ident
    return V


def test_all_requests_finish_with_their_own_result(fake):
    srv = serve.Server({"a": H(), "b": H()}, max_slots=3)
    try:
        rng = np.random.default_rng(0)
        reqs = [srv.submit("ab"[i % 2], _req(int(rng.integers(1, 9)), i)) for i in range(40)]
        for r in reqs:
            r.wait(timeout=30)
    finally:
        srv.close()
    for r in reqs:
        assert np.array_equal(r.I, 2 * r.V)
        assert r.iters == int(r.V[0].real)
        assert r.latency >= r.queue_time >= 0
    for b in fake.opened:
        assert b.max_live <= 3


def test_fifo_admission_per_geometry(fake):
    srv = serve.Server({"a": H()}, max_slots=2)
    try:
        reqs = [srv.submit("a", _req(3, i)) for i in range(12)]
        for r in reqs:
            r.wait(timeout=30)
    finally:
        srv.close()
    assert fake.opened[0].admitted == list(range(12))


def test_hbm_budget_sets_slots(fake):
    per = FakeBatch.bytes(None, 2, 30) - FakeBatch.bytes(None, 1, 30)
    base = FakeBatch.bytes(None, 1, 30) - per
    srv = serve.Server({"a": H(), "b": H()}, hbm_budget=2 * (base + 5 * per), max_slots=64)
    try:
        assert srv.slots("a") == 5 and srv.slots("b") == 5
    finally:
        srv.close()
    srv = serve.Server({"a": H()}, hbm_budget=10 ** 12, max_slots=7)
    try:
        assert srv.slots("a") == 7
    finally:
        srv.close()
    with pytest.raises(MemoryError):
        serve.Server({"a": H()}, hbm_budget=base + per - 1)


def test_engine_error_fails_requests_loudly(fake, monkeypatch):
    def boom(self):
        raise RuntimeError("engine failure")
    monkeypatch.setattr(FakeBatch, "step", boom)
    srv = serve.Server({"a": H()}, max_slots=2)
    r = srv.submit("a", _req(2, 0))
    with pytest.raises(RuntimeError):
        r.wait(timeout=30)
    assert "a" in srv.errors
    with pytest.raises(RuntimeError):
        srv.submit("a", _req(2, 1))
    srv.close()


def test_poisson_arrivals_rate_and_order():
    t = serve.poisson_arrivals(20000, 4.0, seed=1)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.25) < 0.01
    assert np.array_equal(t, serve.poisson_arrivals(20000, 4.0, seed=1))


def test_monostatic_requests_are_transverse_plane_waves():
    class P:
        calls = []

        def plane_wave(self, khat, pol):
            P.calls.append((np.asarray(khat), np.asarray(pol)))
            return np.array([1.0 + 0j])

    out = serve.monostatic_requests(P(), 40, seed=2)
    pols = [p for _, p, _ in out]
    assert pols == [p for _, p, _ in serve.monostatic_requests(P(), 40, seed=2)]
    assert set(pols) == {"VV", "HH"}
    for (phi, pol, _), (k, p) in zip(out, P.calls[:40]):
        assert abs(np.linalg.norm(k) - 1) < 1e-15 and abs(np.linalg.norm(p) - 1) < 1e-15
        assert abs(k @ p) < 1e-15                       # transverse
        assert abs(k[2]) < 1e-15                        # theta = 90 deg
        assert np.allclose(-k[:2], [np.cos(np.deg2rad(phi)), np.sin(np.deg2rad(phi))])
        assert (abs(p[2]) == 1.0) == (pol == "VV")
