"""Pins of the seeded problem builder (mesh, RWG, Eq. 7 entries, octree, Eq. 8 partition,
ACA) against closed forms, invariants, the Mie series and numbers printed in the paper."""
import os

import numpy as np
import pytest

import efie_problem as ep
from efie_problem import mesh, tree
from oracle import krylov, mie, ordering, schur

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, *v = line.split()
            out[k] = [int(x) for x in v]
    return out


# ---- quadrature and closed-form potential integrals ----------------------------------
def test_radon_rule_exact_to_degree_5():
    w, bary = ep.quadrature_rule()
    assert abs(w.sum() - 1.0) < 1e-15
    from math import factorial
    for a in range(6):
        for b in range(6 - a):
            # reference triangle (0,0),(1,0),(0,1): int x^a y^b = a! b! / (a+b+2)!, area 1/2
            x, y = bary[:, 1], bary[:, 2]
            num = 0.5 * np.sum(w * x ** a * y ** b)
            assert abs(num - factorial(a) * factorial(b) / factorial(a + b + 2)) < 1e-15
    x, y = bary[:, 1], bary[:, 2]
    assert abs(0.5 * np.sum(w * x ** 6) - factorial(6) / factorial(8)) > 1e-6   # not degree 6


def _brute_potentials(P, r, levels=6):
    """1/R and (r'-rho)/R integrals by the 7-point rule on 4^levels sub-triangles."""
    w, bary = ep.quadrature_rule()
    tris = [P]
    for _ in range(levels):
        nt = []
        for A, B, C in tris:
            ab, bc, ca = (A + B) / 2, (B + C) / 2, (C + A) / 2
            nt += [(A, ab, ca), (ab, B, bc), (ca, bc, C), (ab, bc, ca)]
        tris = nt
    T = np.array(tris)
    area = 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1)
    Q = np.einsum("qa,tad->tqd", bary, T)
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    rho = r - np.dot(r - P[0], n) * n
    R = np.linalg.norm(Q - r, axis=2)
    s0 = np.sum(area[:, None] * w[None, :] / R)
    sv = np.einsum("t,q,tqd->d", area, w, (Q - rho) / R[..., None])
    return s0, sv


@pytest.mark.parametrize("r", [[0.3, 0.2, 0.4], [1.5, -0.3, 0.1], [0.2, 0.25, 0.05], [-0.4, 0.6, -0.2]])
def test_potential_integrals_off_triangle(r):
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.05]])
    s0, sv = ep.potential_integrals(P, np.array(r))
    b0, bv = _brute_potentials(P, np.array(r), levels=6 if abs(r[2]) > 0.1 else 7)
    assert abs(s0 - b0) / abs(b0) < 1e-7
    assert np.linalg.norm(sv - bv) / np.linalg.norm(bv) < 1e-6


def _polar_potential(P, r, nq=400):
    """In-plane point inside the triangle: int 1/R = sum over the three sub-triangles
    (r, a, b) of int_theta R_edge(theta) d theta (polar coordinates), Gauss-Legendre."""
    x, wq = np.polynomial.legendre.leggauss(nq)
    tot = 0.0
    for i in range(3):
        a, b = P[i], P[(i + 1) % 3]
        u, v = a - r, b - r
        th = np.arccos(np.clip(np.dot(u, v) / np.linalg.norm(u) / np.linalg.norm(v), -1, 1))
        h = np.linalg.norm(np.cross(b - a, r - a)) / np.linalg.norm(b - a)   # distance to the edge line
        phi0 = np.arccos(np.clip(h / np.linalg.norm(u), -1, 1))
        # angle measured from the foot of the perpendicular: R(theta) = h / cos(theta - phi_foot)
        sgn = np.sign(np.dot(np.cross(u, b - a), np.cross(u, v)))
        t = 0.5 * th * (x + 1)
        # parametrise from u towards v; angle to the perpendicular foot along u is phi0 (signed)
        ang = phi0 - t if sgn >= 0 else phi0 + t
        R = h / np.cos(ang)
        tot += 0.5 * th * np.sum(wq * R)
    return tot


def test_potential_integral_singular_in_plane():
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.8, 0.0]])
    for r in ([0.4, 0.3, 0.0], [0.25, 0.1, 0.0], [0.5, 0.05, 0.0]):
        s0, _ = ep.potential_integrals(P, np.array(r))
        ref = _polar_potential(P, np.array(r))
        assert abs(s0 - ref) / ref < 1e-10


# ---- meshes and RWG -----------------------------------------------------------------
@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_icosphere_counts_and_euler(d):
    V, T = mesh.icosphere(d, 1.0)
    rwg = mesh.RWG(V, T)
    assert len(T) == 20 * 4 ** d and rwg.n == 30 * 4 ** d
    assert len(V) - rwg.n + len(T) == 2
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0)


def test_plate_counts_and_jitter():
    V, T = mesh.plate(10, 1.0, jitter=0.1, seed=0)
    rwg = mesh.RWG(V, T)
    assert rwg.n == 3 * 10 ** 2 - 2 * 10
    V0, _ = mesh.plate(10, 1.0, jitter=0.0)
    d = np.abs(V - V0).max(axis=1)
    assert d.max() <= 0.1 * 0.1 + 1e-15
    onb = (np.isclose(V0[:, 0], 0) | np.isclose(V0[:, 0], 1) | np.isclose(V0[:, 1], 0) | np.isclose(V0[:, 1], 1))
    assert np.all(d[onb] == 0)


def test_rwg_normal_flux_continuity():
    V, T = mesh.icosphere(1, 1.0)
    rwg = mesh.RWG(V, T)
    for n in range(rwg.n):
        a, b = V[rwg.edge[n, 0]], V[rwg.edge[n, 1]]
        mid = 0.5 * (a + b)
        e = (b - a) / np.linalg.norm(b - a)
        fl = []
        for s, sign in ((0, 1.0), (1, -1.0)):
            t = rwg.tri[n, s]
            P = V[T[t]]
            A = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
            f = sign * rwg.length[n] / (2 * A) * (mid - V[rwg.free[n, s]])
            # normal to the edge inside the triangle plane, pointing from T+ to T-
            nt = np.cross(P[1] - P[0], P[2] - P[0])
            m = np.cross(e, nt / np.linalg.norm(nt))
            if np.dot(m, mid - V[rwg.free[n, 0]]) < 0:
                m = -m
            fl.append(np.dot(f, m))
        assert abs(fl[0] - 1.0) < 1e-12 and abs(fl[1] - 1.0) < 1e-12


# ---- cluster tree and partition -------------------------------------------------------
def test_plate_level2_leaf_sizes_match_table5():
    """Table 5 lists 363- and 385-row/column fill blocks for the 5985-unknown plate at
    oct-tree level 2: the midpoint octree reproduces exactly those leaf sizes."""
    g = golden("paper_plate_5985.txt")
    V, T = mesh.plate(45, 5.0, jitter=0.0)
    rwg = mesh.RWG(V, T)
    assert rwg.n == 5985
    root, leaves, perm = tree.build_tree(rwg.midpoints(), vertices=V, fixed_level=2)
    sizes = sorted(lf.hi - lf.lo for lf in leaves)
    assert sizes.count(363) == 9 and sizes.count(385) == 6 and sizes.count(408) == 1
    assert set(g["table5_block_sizes"]) <= set(sizes)


def test_plate_level2_table6_nnz_is_a_full_block_triangle():
    """Table 6's level-2 "no compression" count equals, within 0.3%, the full block lower
    triangle (plus the identity diagonal) on the 16 leaves of this octree, whose sizes Table 5
    fixes: at level 2 the paper's fill is complete.  The near field read here (Eq. 8 with
    eta = 1) fills 85-100% of that triangle -- the narrower level-2 near field of reading 4;
    at level 3, where the fill is partial, the counts agree (next test)."""
    g = golden("paper_plate_5985.txt")
    V, T = mesh.plate(45, 5.0, jitter=0.0)
    rwg = mesh.RWG(V, T)
    root, leaves, perm = tree.build_tree(rwg.midpoints(), vertices=V, fixed_level=2)
    blo, bhi = rwg.support_boxes()
    tree.attach_boxes(root, perm, blo, bhi)
    near, far = tree.partition(root, 1.0)
    nl = len(leaves)
    sz = np.array([lf.hi - lf.lo for lf in leaves])
    full = sum(int(sz[k] * sz[j]) for k in range(nl) for j in range(k + 1, nl)) + rwg.n
    ref = g["table6_nnz_level2_uncompressed"][0]
    assert abs(full - ref) / ref < 0.003
    S = schur.symbolic_fill(nl, sorted({(min(a, b), max(a, b)) for a, b in near}))
    nnz = sum(int(sz[k] * sz[j]) for k in range(nl) for j in S[k]) + rwg.n
    assert 0.85 * full <= nnz <= full


def test_plate_level3_fill_nnz_matches_table6():
    """Uncompressed scaling-coefficient NNZ (Table 6, oct-tree 3, no ordering) within 3%."""
    g = golden("paper_plate_5985.txt")
    V, T = mesh.plate(45, 5.0, jitter=0.0)
    rwg = mesh.RWG(V, T)
    root, leaves, perm = tree.build_tree(rwg.midpoints(), vertices=V, fixed_level=3)
    blo, bhi = rwg.support_boxes()
    tree.attach_boxes(root, perm, blo, bhi)
    near, far = tree.partition(root, 1.0)
    nl = len(leaves)
    sz = np.array([lf.hi - lf.lo for lf in leaves])
    S = schur.symbolic_fill(nl, sorted({(min(a, b), max(a, b)) for a, b in near}))
    nnz = sum(int(sz[k] * sz[j]) for k in range(nl) for j in S[k]) + rwg.n
    ref = g["table6_nnz_level3_uncompressed"][0]
    assert abs(nnz - ref) / ref < 0.03


def test_partition_covers_every_entry_once(sphere480):
    P = sphere480
    n = P.n
    cover = np.zeros((n, n), dtype=np.int32)
    lp = P.leaf_ptr
    for t, s in zip(P.near_t, P.near_s):
        cover[lp[t]:lp[t + 1], lp[s]:lp[s + 1]] += 1
        if t != s:
            cover[lp[s]:lp[s + 1], lp[t]:lp[t + 1]] += 1
    for b in range(len(P.far_rank)):
        r0, r1, c0, c1 = P.far_r0[b], P.far_r1[b], P.far_c0[b], P.far_c1[b]
        assert r1 <= c0
        cover[r0:r1, c0:c1] += 1
        cover[c0:c1, r0:r1] += 1
    assert np.all(cover == 1)
    assert sorted(P.perm.tolist()) == list(range(n))
    assert np.all(np.diff(P.leaf_ptr) <= 32)


def test_touching_supports_are_near(sphere1920):
    P = sphere1920
    rwg = P.rwg
    pos = np.empty(P.n, dtype=np.int64)
    pos[P.perm] = np.arange(P.n)
    leaf_of = np.searchsorted(P.leaf_ptr, pos, side="right") - 1
    near = set(zip(P.near_t.tolist(), P.near_s.tolist()))
    tri_sets = [set(rwg.tri[i]) for i in range(P.n)]
    verts = [set(rwg.T[list(tri_sets[i])].ravel()) for i in range(P.n)]
    rng = np.random.default_rng(0)
    for i in rng.choice(P.n, 200, replace=False):
        for j in range(P.n):
            if verts[i] & verts[j]:
                a, b = sorted((int(leaf_of[i]), int(leaf_of[j])))
                assert (a, b) in near


# ---- EFIE entries ---------------------------------------------------------------------
def test_entries_symmetric_and_mirrored(sphere480):
    P = sphere480
    ev = ep.EntryEvaluator(P.rwg)
    Z = ev.dense()
    assert np.linalg.norm(Z - Z.T) / np.linalg.norm(Z) < 1e-3
    # stored diagonal near blocks are exactly symmetric
    lp = P.leaf_ptr
    for b in range(len(P.near_t)):
        if P.near_t[b] == P.near_s[b]:
            m = lp[P.near_t[b] + 1] - lp[P.near_t[b]]
            B = P.near_data[P.near_off[b]:P.near_off[b] + m * m].reshape(m, m).T
            assert np.array_equal(B, B.T)


def test_hmatrix_close_to_dense(sphere1920):
    P = sphere1920
    ev = ep.EntryEvaluator(P.rwg)
    Z = ev.dense()
    Zs = np.triu(Z) + np.triu(Z, 1).T
    F = schur.setup(P, np.arange(len(P.leaf_ptr) - 1), 0.0)
    S = krylov.System(P, F)
    X = np.random.default_rng(1).standard_normal((P.n, 4))
    err = max(np.linalg.norm(S.Z_orig(X[:, c]) - Zs @ X[:, c]) / np.linalg.norm(Zs @ X[:, c]) for c in range(4))
    assert err < 10 * 1e-3


def test_plane_wave_linear_in_polarisation(sphere480):
    P = sphere480
    a = P.plane_wave([0, 0, -1], [1, 0, 0])
    b = P.plane_wave([0, 0, -1], [0, 1, 0])
    c = P.plane_wave([0, 0, -1], [2, -3, 0])
    assert np.linalg.norm(c - (2 * a - 3 * b)) < 1e-12 * np.linalg.norm(c)


# ---- Mie series -----------------------------------------------------------------------
def test_mie_rayleigh_limit():
    for ka in (0.01, 0.03):
        a = ka / (2 * np.pi)
        assert abs(mie.monostatic(ka) / (9 * np.pi * a * a * ka ** 4) - 1) < 2 * ka ** 2


def test_mie_bistatic_backscatter_equals_monostatic():
    for ka in (0.5, 3.77, 15.0):
        sE, sH = mie.bistatic(ka, np.array([np.pi]))
        m = mie.monostatic(ka)
        assert abs(sE[0] - m) < 1e-10 * m and abs(sH[0] - m) < 1e-10 * m


def test_sphere_rcs_matches_mie(sphere1920):
    """1920-unknown PEC sphere, a = 0.6 lambda: E- and H-plane bistatic RCS within 0.5 dB
    of the Mie series (angles within 20 dB of the cut maximum)."""
    P = sphere1920
    F = schur.setup(P, ordering.rcm(len(P.leaf_ptr) - 1, list(zip(P.near_t.tolist(), P.near_s.tolist()))), 0.0)
    S = krylov.System(P, F)
    b = P.plane_wave([0, 0, -1], [1, 0, 0])
    x, it, rr, ok = krylov.solve(S, b, tol=1e-8, restart=30)
    assert ok
    th = np.linspace(0, np.pi, 91)
    rE = np.stack([np.sin(th), 0 * th, -np.cos(th)], 1)
    rH = np.stack([0 * th, np.sin(th), -np.cos(th)], 1)
    sE, sH = ep.bistatic_rcs(P.rwg, x, rE), ep.bistatic_rcs(P.rwg, x, rH)
    mE, mH = mie.bistatic(2 * np.pi * 0.6, th)
    for s, m in ((sE, mE), (sH, mH)):
        keep = m > m.max() * 1e-2
        assert np.max(np.abs(10 * np.log10(s[keep] / m[keep]))) < 0.5
