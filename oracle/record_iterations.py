"""Records the oracle's own GMRES iteration counts on the benchmark workloads (test
infrastructure: the CPU-baseline leg of the benchmark reads them, so that its per-RHS
solve cost uses the oracle's count and not the GPU's).

For each entry: the problem is built by ``efie_problem`` (the seeded input generator), the
oracle orders it (Algorithm 1, RCM), factors it (Sec. 3.1-3.4 with fill_tol) and solves the
Eq. 28 system with GMRES(restart) to the preconditioned tolerance for the listed right-hand
sides: monostatic plane waves at theta = 90 deg, azimuth phi (deg), theta-hat (VV)
polarisation, i.e. the benchmark's k = -(cos phi, sin phi, 0), p = (0, 0, -1); or, for the
1,920-unknown sphere, the single wave k = -z, p = x.  Wall times of the oracle's setup and
solves (one BLAS thread) are stored beside the counts.

    python oracle/record_iterations.py [name ...]      # default: sphere1920 sphere30720

writes oracle/iterations.json (merged with what is already there).  Only oracle/ and the
input generator are used.
"""
import json
import os
import sys
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

OUT = os.path.join(HERE, "iterations.json")

# workload -> (fill_tol, tol, restart, right-hand sides: list of phi in degrees, or "z")
CASES = {
    "sphere1920": (1e-2, 1e-4, 30, ["z"]),
    "sphere30720": (1e-2, 1e-4, 30, [0.0, 90.0]),
}


def key(name, fill_tol, tol, restart):
    return "%s fill_tol=%g tol=%g restart=%d" % (name, fill_tol, tol, restart)


def rhs(P, spec):
    if spec == "z":
        return P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    ph = np.deg2rad(spec)
    return P.plane_wave([-np.cos(ph), -np.sin(ph), 0.0], [0.0, 0.0, -1.0])


def record(name):
    import efie_problem as ep
    from oracle import krylov, ordering, schur
    fill_tol, tol, restart, specs = CASES[name]
    P = ep.build(name)
    t0 = time.perf_counter()
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    F = schur.setup(P, order, fill_tol=fill_tol)
    S = krylov.System(P, F)
    t_setup = time.perf_counter() - t0
    its, secs = [], []
    for spec in specs:
        t1 = time.perf_counter()
        _, it, rr, ok = krylov.solve(S, rhs(P, spec), tol=tol, restart=restart)
        secs.append(time.perf_counter() - t1)
        if not ok:
            raise RuntimeError("oracle GMRES did not converge on %s (%s)" % (name, spec))
        its.append(int(it))
    return key(name, fill_tol, tol, restart), {
        "workload": name, "n": int(P.n), "fill_tol": fill_tol, "tol": tol, "restart": restart,
        "rhs": [("k=-z, p=x" if s == "z" else "theta 90 deg, phi %g deg, VV" % s) for s in specs],
        "iters": its, "oracle_setup_s": t_setup, "oracle_solve_s": secs, "blas_threads": 1}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        k, v = record(name)
        data[k] = v
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")
        print(k, v["iters"], "setup %.1f s" % v["oracle_setup_s"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
