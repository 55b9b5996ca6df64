"""The H-matrix inputs of the solve built on the GPU (Sec. 2): mesh, RWG functions, cluster
tree and admissible partition (Eq. 8) come from the seeded input generator; the near-field
blocks (Eq. 7) and the far-field ACA factors (Eqs. 9-10) are computed by hm_efie_fill and
hm_efie_far.  The result has the layout of ``efie_problem.builder.Problem``, so it goes to
``hmat_create`` unchanged; ``timings`` reports the matrix setup time t_sm of Eq. 46."""
import time

import numpy as np

from efie_problem import builder as _b
from efie_problem import mesh as _mesh
from efie_problem import tree as _tree

from . import hmsolve as H


def build_problem(spec, device=0):
    """Returns (problem, timings): timings in seconds for the geometry (mesh, tree, partition
    on the host), the near field and the far field (each a GPU call including its transfers)."""
    if isinstance(spec, str):
        spec = _b.SPECS[spec]
    t0 = time.perf_counter()
    V, T = _b.make_mesh(spec)
    rwg = _mesh.RWG(V, T)
    root, leaves, perm = _tree.build_tree(rwg.midpoints(), spec.get("leaf", 64), vertices=V,
                                          fixed_level=spec.get("level"))
    blo, bhi = rwg.support_boxes()
    _tree.attach_boxes(root, perm, blo, bhi)
    near, far = _tree.partition(root, spec.get("eta", 1.0))
    leaf_ptr = np.array([lf.lo for lf in leaves] + [leaves[-1].hi], dtype=np.int64)
    mesh = H.Mesh(rwg.V, rwg.T, rwg.tri, rwg.free, _b.K0, _b.ETA0)
    P = _b.Problem()
    P.rwg, P.k, P.eta0 = rwg, _b.K0, _b.ETA0
    P.perm = perm.astype(np.int32)
    P.leaf_ptr = leaf_ptr.astype(np.int32)
    nr = sorted({(min(t, s), max(t, s)) for t, s in near})
    P.near_t = np.array([a for a, _ in nr], dtype=np.int32)
    P.near_s = np.array([b for _, b in nr], dtype=np.int32)
    rows = [perm[leaf_ptr[t]:leaf_ptr[t + 1]] for t, _ in nr]
    cols = [perm[leaf_ptr[s]:leaf_ptr[s + 1]] for _, s in nr]
    fr = [(t, s) for t, s in far if t.lo < s.lo]
    fr.sort(key=lambda ts: (ts[0].lo, ts[1].lo, ts[0].hi, ts[1].hi))
    rl = [perm[t.lo:t.hi] for t, _ in fr]
    cl = [perm[s.lo:s.hi] for _, s in fr]
    t1 = time.perf_counter()
    data, off = H.hm_efie_fill(mesh, rows, cols, mirror=1, device=device)
    P.near_off = off[:-1].astype(np.int64)
    P.near_data = data
    t2 = time.perf_counter()
    if fr:
        rank, uoff, voff, U, Vf = H.hm_efie_far(mesh, rl, cl, spec.get("aca_eps", 1e-3), device=device)
    else:
        rank, uoff, voff = (np.zeros(0, np.int32), np.zeros(0, np.int64), np.zeros(0, np.int64))
        U, Vf = np.zeros(0, np.complex128), np.zeros(0, np.complex128)
    t3 = time.perf_counter()
    P.far_r0 = np.array([t.lo for t, _ in fr], dtype=np.int32)
    P.far_r1 = np.array([t.hi for t, _ in fr], dtype=np.int32)
    P.far_c0 = np.array([s.lo for _, s in fr], dtype=np.int32)
    P.far_c1 = np.array([s.hi for _, s in fr], dtype=np.int32)
    P.far_rank = rank.astype(np.int32)
    P.far_uoff = uoff.astype(np.int64)
    P.far_voff = voff.astype(np.int64)
    P.far_U = U
    P.far_V = Vf
    P.spec = dict(spec)
    return P, {"geometry_s": t1 - t0, "near_s": t2 - t1, "far_s": t3 - t2, "matrix_s": t3 - t1}
