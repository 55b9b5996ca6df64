"""Serving loop over resident geometries: continuous batching of solve requests.

Each geometry keeps its H-matrix and factored preconditioner resident on the device (one
handle, one CUDA stream) and one slot engine (``hmsolve.Batch``, the hm_batch_* calls of
libhmsolve.so).  A driver thread per geometry admits queued requests into free slots at
every engine step, so requests that arrive while others are in flight join the running
multi-column GMRES as soon as a slot frees up, and the geometries' steps overlap on the
GPU through their streams.  The number of slots per geometry is what the HBM budget
affords.  Every request records its submit, admit and finish times.

The paper (Sec. 5) solves many right-hand sides per geometry (monostatic sweeps); this
module only schedules those solves, the arithmetic is the library's.
"""
import threading
import time
from collections import deque

import numpy as np

from . import hmsolve


class Request:
    """A solve request; ``wait()`` blocks until it has finished.

    After completion: ``I`` (complex128 (n,), original RWG order), ``iters``, ``relres``,
    ``status`` (HM_OK / HM_ENOCONV), ``latency`` = finish - submit in seconds,
    ``queue_time`` = admit - submit."""

    def __init__(self, geom, V, tol, maxit, tag=None):
        self.geom, self.V, self.tol, self.maxit, self.tag = geom, V, tol, maxit, tag
        self.t_submit = self.t_admit = self.t_done = None
        self.I = None
        self.iters = self.relres = self.status = None
        self.error = None
        self._ev = threading.Event()

    def done(self):
        return self._ev.is_set()

    def wait(self, timeout=None):
        if not self._ev.wait(timeout):
            raise TimeoutError("request not finished")
        if self.error is not None:
            raise self.error
        return self.I

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_submit

    @property
    def queue_time(self):
        return None if self.t_admit is None else self.t_admit - self.t_submit


class _Geometry:
    def __init__(self, name, h, slots, restart, tol, maxit):
        self.name, self.h = name, h
        self.tol, self.maxit = tol, maxit
        self.batch = hmsolve.Batch(h, slots, restart)
        self.slots = slots
        self.queue = deque()
        self.inflight = {}
        self.cv = threading.Condition()
        self.steps = 0
        self.busy_s = 0.0
        self.thread = None


class Server:
    """``Server({name: handle}, hbm_budget=bytes)``: handles already through precond_setup.

    ``hbm_budget`` bounds the device bytes of all slot engines together (split evenly over
    the geometries); ``max_slots`` caps the slots per geometry (the multi-column width of its
    operator launches).  ``submit(name, V)`` returns a Request at once; ``close()`` stops the
    driver threads after the queues have drained."""

    def __init__(self, geometries, hbm_budget=None, max_slots=64, restart=30, tol=1e-4, maxit=5000,
                 restarts=None):
        self.geoms = {}
        self.errors = {}
        share = None if hbm_budget is None else hbm_budget // max(1, len(geometries))
        for name, h in geometries.items():
            r = (restarts or {}).get(name, restart)
            slots = max_slots
            if share is not None:
                per = hmsolve.Batch.bytes(h, 2, r) - hmsolve.Batch.bytes(h, 1, r)
                base = hmsolve.Batch.bytes(h, 1, r) - per
                slots = int(min(max_slots, max(0, (share - base) // per)))
                if slots < 1:
                    raise MemoryError("HBM budget too small for one slot of geometry %r" % name)
            self.geoms[name] = _Geometry(name, h, slots, r, tol, maxit)
        self._stop = False
        for g in self.geoms.values():
            g.thread = threading.Thread(target=self._drive, args=(g,), daemon=True, name="hm-serve-" + g.name)
            g.thread.start()

    def slots(self, name):
        return self.geoms[name].slots

    def submit(self, name, V, tol=None, maxit=None, tag=None):
        if name in self.errors:
            raise RuntimeError("geometry %r failed: %s" % (name, self.errors[name]))
        g = self.geoms[name]
        req = Request(name, np.ascontiguousarray(V, dtype=np.complex128), g.tol if tol is None else tol,
                      g.maxit if maxit is None else maxit, tag)
        req.t_submit = time.perf_counter()
        with g.cv:
            g.queue.append(req)
            g.cv.notify()
        return req

    def _drive(self, g):
        b = g.batch
        try:
            while True:
                with g.cv:
                    while not g.queue and not g.inflight and not self._stop:
                        g.cv.wait()
                    if self._stop and not g.queue and not g.inflight:
                        return
                    pending = []
                    while g.queue and len(g.inflight) + len(pending) < g.slots:
                        pending.append(g.queue.popleft())
                for req in pending:   # admission: a free slot per request
                    slot = b.submit(req.V, req.tol, req.maxit)
                    if slot is None:
                        with g.cv:
                            g.queue.appendleft(req)
                        continue
                    req.t_admit = time.perf_counter()
                    g.inflight[slot] = req
                t0 = time.perf_counter()
                fin = b.step()
                g.busy_s += time.perf_counter() - t0
                g.steps += 1
                for slot in fin:
                    req = g.inflight.pop(slot)
                    req.I, req.iters, req.relres, req.status = b.result(slot)
                    req.t_done = time.perf_counter()
                    req._ev.set()
        except Exception as exc:   # fail every request of this geometry loudly
            with g.cv:
                self.errors[g.name] = exc
                rest = list(g.inflight.values()) + list(g.queue)
                g.inflight.clear()
                g.queue.clear()
            for req in rest:
                req.error = exc
                req._ev.set()

    def close(self):
        self._stop = True
        for g in self.geoms.values():
            with g.cv:
                g.cv.notify_all()
        for g in self.geoms.values():
            if g.thread is not None:
                g.thread.join()
            g.batch.close()


def monostatic_requests(prob, count, seed, phi_step_deg=1.0, plane="xy"):
    """Right-hand sides of a monostatic sweep: observation directions at phi = 0, 1, ... deg in
    the xy plane (theta = 90 deg), the polarisation theta-hat (VV) or phi-hat (HH) drawn per
    request from a seeded generator.  plane="xz" sweeps the same angles in the xz plane
    (direction (cos phi, 0, sin phi), VV in that plane, HH = y-hat): for a plate in the xy
    plane this is the horizontal sweep of the same plate standing upright.
    Returns a list of (phi_deg, pol, V)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        phi = np.deg2rad(i * phi_step_deg)
        if plane == "xy":
            rhat = np.array([np.cos(phi), np.sin(phi), 0.0])
            pv, ph = np.array([0.0, 0.0, -1.0]), np.array([-np.sin(phi), np.cos(phi), 0.0])
        else:
            rhat = np.array([np.cos(phi), 0.0, np.sin(phi)])
            pv, ph = np.array([-np.sin(phi), 0.0, np.cos(phi)]), np.array([0.0, 1.0, 0.0])
        khat = -rhat                                     # incident from the observation direction
        pol = "VV" if rng.integers(2) == 0 else "HH"
        out.append((i * phi_step_deg, pol, prob.plane_wave(khat, pv if pol == "VV" else ph)))
    return out


def poisson_arrivals(count, rate, seed):
    """Arrival times (s, from 0) of a Poisson stream of ``count`` requests at ``rate``/s."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def run_stream(server, streams):
    """Submits each request at its arrival time.  streams: list of (name, arrivals, rhs list).
    Returns the Request objects in submission order once all have finished."""
    events = sorted(((t, name, V) for name, arr, rhs in streams for t, V in zip(arr, rhs)), key=lambda e: e[0])
    t0 = time.perf_counter()
    reqs = []
    for t, name, V in events:
        dt = t0 + t - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        reqs.append(server.submit(name, V))
    for r in reqs:
        r.wait()
    return reqs


def latency_summary(reqs):
    lat = np.array([r.latency for r in reqs])
    return {"requests": len(reqs), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
