"""Pins of the CPU oracle (ordering, symmetric Schur preconditioner, GMRES) against the
paper's 4-block example (Sec. 3.1, Fig. 2, Eqs. 12-21), brute-force dense linear algebra,
closed-form special cases and stated invariants."""
from types import SimpleNamespace

import numpy as np
import pytest
import scipy.sparse as ssp
import scipy.sparse.csgraph as csg

from oracle import krylov, ordering, schur


def rand_sym(n, rng):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return A + A.T


def block_problem(sizes, pairs, rng, far=None, diag_boost=4.0):
    """Problem-like object: complex-symmetric near blocks on ``pairs`` (t <= s), leaves in
    order, optional far blocks given as dense (t, s) -> matrix stored with rank -1."""
    lp = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(lp[-1])
    Z = np.zeros((n, n), dtype=np.complex128)
    for t, s in pairs:
        m, k = sizes[t], sizes[s]
        B = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
        if t == s:
            B = B + B.T + diag_boost * np.sqrt(m) * np.eye(m)
        Z[lp[t]:lp[t + 1], lp[s]:lp[s + 1]] = B
        Z[lp[s]:lp[s + 1], lp[t]:lp[t + 1]] = B.T
    offs, data = [], []
    o = 0
    for t, s in pairs:
        B = Z[lp[t]:lp[t + 1], lp[s]:lp[s + 1]]
        offs.append(o)
        data.append(B.ravel(order="F"))
        o += B.size
    p = SimpleNamespace(leaf_ptr=lp, perm=np.arange(n, dtype=np.int32),
                        near_t=np.array([a for a, _ in pairs], np.int32), near_s=np.array([b for _, b in pairs], np.int32),
                        near_off=np.array(offs, np.int64), near_data=np.concatenate(data))
    ZF = np.zeros_like(Z)
    fr = far or []
    fU, fo = [], []
    uo = 0
    for (t, s), B in fr:
        ZF[lp[t]:lp[t + 1], lp[s]:lp[s + 1]] = B
        ZF[lp[s]:lp[s + 1], lp[t]:lp[t + 1]] = B.T
        fU.append(B.ravel(order="F"))
        fo.append(uo)
        uo += B.size
    p.far_r0 = np.array([lp[t] for (t, s), _ in fr], np.int32)
    p.far_r1 = np.array([lp[t + 1] for (t, s), _ in fr], np.int32)
    p.far_c0 = np.array([lp[s] for (t, s), _ in fr], np.int32)
    p.far_c1 = np.array([lp[s + 1] for (t, s), _ in fr], np.int32)
    p.far_rank = -np.ones(len(fr), np.int32)
    p.far_uoff = np.array(fo, np.int64)
    p.far_voff = np.zeros(len(fr), np.int64)
    p.far_U = np.concatenate(fU) if fU else np.zeros(0, np.complex128)
    p.far_V = np.zeros(0, np.complex128)
    return p, Z, ZF


# ---- Sec. 3.1, Fig. 2: the four-block worked example ------------------------------------
def test_four_block_example_eqs_12_to_21():
    rng = np.random.default_rng(0)
    sizes = [3, 4, 2, 5]
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]   # blocks 1, 4 far
    p, Z, _ = block_problem(sizes, pairs, rng)
    lp = p.leaf_ptr
    sl = [slice(lp[k], lp[k + 1]) for k in range(4)]
    n = Z.shape[0]
    Zb = lambda M, i, j: M[sl[i], sl[j]]
    # Eq. 14 / 16: right and left scaling coefficients of block 1, from their own formulas
    a1 = np.eye(n, dtype=complex)
    al1 = np.eye(n, dtype=complex)
    Z11i = np.linalg.inv(Zb(Z, 0, 0))
    for j in (1, 2):
        a1[sl[0], sl[j]] = -Z11i @ Zb(Z, 0, j)
        al1[sl[j], sl[0]] = -Zb(Z, j, 0) @ Z11i
    assert np.allclose(al1, a1.T, atol=1e-13)                   # Sec. 3.2: alpha' = alpha^T
    Z1 = al1 @ Z @ a1                                            # Eq. 18
    # Eq. 19: first block row/column decoupled, (2,4) untouched, Schur complements elsewhere
    nrm = np.linalg.norm(Z)
    for j in (1, 2, 3):
        assert np.linalg.norm(Zb(Z1, 0, j)) < 1e-13 * nrm and np.linalg.norm(Zb(Z1, j, 0)) < 1e-13 * nrm
    assert np.allclose(Zb(Z1, 1, 3), Zb(Z, 1, 3), rtol=0, atol=1e-13 * nrm)
    for i in (1, 2):
        for j in (1, 2):
            ref = Zb(Z, i, j) - Zb(Z, i, 0) @ Z11i @ Zb(Z, 0, j)
            assert np.linalg.norm(Zb(Z1, i, j) - ref) < 1e-12 * nrm
    # Eqs. 20-21 with the oracle's factorisation: blockdiag(D_k) exactly
    F = schur.setup(p, np.arange(4), fill_tol=0.0)
    assert F.S == [[1, 2], [2, 3], [3], []]                     # no fill at (2,4) from step 1
    L, D = schur.ldlt_dense(F)
    Linv = np.linalg.inv(L)
    Zt = Linv @ Z @ Linv.T                                       # alpha'_3 alpha'_2 alpha'_1 Z alpha_1 alpha_2 alpha_3
    for i in range(4):
        for j in range(4):
            blk = Zb(Zt, i, j)
            if i == j:
                assert np.linalg.norm(blk - F.D[i]) < 1e-12 * nrm
            else:
                assert np.linalg.norm(blk) < 1e-12 * nrm
    assert np.linalg.norm(F.D[0] - Zb(Z, 0, 0)) == 0             # D_1 = Z_11 (Eq. 21)


def test_schur_blocks_equal_dense_schur_complements(sphere480):
    P = sphere480
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    F = schur.setup(P, order, 0.0)
    S = krylov.System(P, F)
    A = schur.near_blocks_in_order(P, order)
    off = S.off
    Zn = np.zeros((S.n, S.n), dtype=np.complex128)
    for (i, j), B in A.items():
        Zn[off[i]:off[i + 1], off[j]:off[j + 1]] = B
        Zn[off[j]:off[j + 1], off[i]:off[i + 1]] = B.T
    for k in [0, 1, nl // 3, nl // 2, nl - 2, nl - 1]:
        a, b = off[k], off[k + 1]
        ref = Zn[a:b, a:b] - Zn[a:b, :a] @ np.linalg.solve(Zn[:a, :a], Zn[:a, a:b]) if a else Zn[a:b, a:b]
        assert np.linalg.norm(F.D[k] - ref) / np.linalg.norm(ref) < 1e-10
    L, D = schur.ldlt_dense(F)
    assert np.linalg.norm(L @ D @ L.T - Zn) / np.linalg.norm(Zn) < 1e-12


def test_symbolic_fill_equals_dense_factor_pattern():
    rng = np.random.default_rng(5)
    nb = 12
    sizes = [2] * nb
    pairs = sorted({(min(a, b), max(a, b)) for a, b in
                    [(i, i) for i in range(nb)] + [tuple(rng.choice(nb, 2, replace=False)) for _ in range(14)]})
    p, Z, _ = block_problem(sizes, pairs, rng)
    F = schur.setup(p, np.arange(nb), 0.0)
    L, D = schur.ldlt_dense(F)
    for k in range(nb):
        nz = [j for j in range(k + 1, nb) if np.linalg.norm(L[2 * j:2 * j + 2, 2 * k:2 * k + 2]) > 1e-12]
        assert nz == F.S[k]


def test_fill_compression():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((30, 4)) + 1j * rng.standard_normal((30, 4))
    Y = rng.standard_normal((4, 30)) + 1j * rng.standard_normal((4, 30))
    W = X @ Y + 1e-4 * (rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30)))
    Wc, r = schur.compress_block(W, 1e-2)
    assert r == 4
    assert np.linalg.norm(W - Wc) <= 1e-2 * np.linalg.norm(W)
    Wc3, r3 = schur.compress_block(W[:, :3] @ np.ones((3, 30)), 1e-2)
    assert r3 == -1 or r3 <= 3
    full = rng.standard_normal((6, 6)) + 0j
    assert schur.compress_block(full, 1e-2)[1] == -1            # dense is cheaper


def test_compression_zero_tolerance_is_exact(sphere480):
    P = sphere480
    order = np.arange(len(P.leaf_ptr) - 1)
    F0 = schur.setup(P, order, 0.0)
    F1 = schur.setup(P, order, 1e-2)
    assert F1.rank and all(np.array_equal(F0.D[k], F1.D[k]) for k in range(F0.nb))
    for key, r in F1.rank.items():
        W = F1.W[key]
        assert np.linalg.norm(F1.Wc[key] - W) <= 1e-2 * np.linalg.norm(W) * (1 + 1e-12)
        assert key[1] > key[0] and (key[1], key[0]) not in F1.near_pairs
    assert schur.nnz_coefficients(F1) <= schur.nnz_coefficients(F0)


# ---- GMRES --------------------------------------------------------------------------------
def test_givens_rotation():
    for a, b in [(1 + 2j, 3 - 1j), (0.0, 2 + 1j), (1e-3j, 5.0)]:
        c, s, rho = krylov.givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        v = G @ np.array([a, b])
        assert abs(v[1]) < 1e-14 * abs(rho) and abs(v[0] - rho) < 1e-14 * abs(rho)
        assert np.allclose(G @ G.conj().T, np.eye(2), atol=1e-14)


def test_gmres_full_space_equals_direct_solve():
    rng = np.random.default_rng(4)
    n = 40
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    hist = []
    x, it, rr, ok = krylov.gmres(lambda v: A @ v, c, 1e-12, n, hist=hist)
    assert ok and it <= n
    assert np.linalg.norm(x - np.linalg.solve(A, c)) / np.linalg.norm(x) < 1e-10
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))


def test_gmres_restart_estimate_equals_true_residual():
    rng = np.random.default_rng(6)
    n = 60
    A = np.eye(n) * 20 + rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    c = rng.standard_normal(n) + 0j
    hist = []
    x, it, rr, ok = krylov.gmres(lambda v: A @ v, c, 1e-9, 7, hist=hist)
    assert ok and it > 7                                          # restarted at least once
    true = np.linalg.norm(c - A @ x) / np.linalg.norm(c)
    assert abs(true - rr) <= 1e-10 + 1e-6 * rr


def test_no_far_field_converges_in_one_step():
    """With Z_F = 0 the preconditioned operator of Eq. 28 is the identity: one Arnoldi
    step, and the solution is the dense solve of Z_N."""
    rng = np.random.default_rng(8)
    sizes = [3, 5, 4, 2, 6]
    pairs = [(0, 0), (0, 1), (1, 1), (1, 2), (2, 2), (2, 3), (3, 3), (3, 4), (4, 4), (0, 4)]
    p, Z, _ = block_problem(sizes, pairs, rng)
    F = schur.setup(p, np.array([2, 0, 4, 1, 3]), 0.0)
    S = krylov.System(p, F)
    b = rng.standard_normal(Z.shape[0]) + 1j * rng.standard_normal(Z.shape[0])
    x, it, rr, ok = krylov.solve(S, b, tol=1e-12, restart=10)
    assert ok and it == 1
    assert np.linalg.norm(x - np.linalg.solve(Z, b)) / np.linalg.norm(x) < 1e-12


def test_far_field_system_solution_equals_dense():
    rng = np.random.default_rng(9)
    sizes = [3, 5, 4, 2, 6]
    pairs = [(0, 0), (0, 1), (1, 1), (1, 2), (2, 2), (2, 3), (3, 3), (3, 4), (4, 4)]
    far = [((0, 2), 0.3 * (rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4)))),
           ((1, 4), 0.3 * (rng.standard_normal((5, 6)) + 1j * rng.standard_normal((5, 6))))]
    p, Z, ZF = block_problem(sizes, pairs, rng, far=far)
    F = schur.setup(p, ordering.rcm(5, pairs), 0.0)
    S = krylov.System(p, F)
    b = rng.standard_normal(Z.shape[0]) + 1j * rng.standard_normal(Z.shape[0])
    x, it, rr, ok = krylov.solve(S, b, tol=1e-13, restart=20)
    assert ok
    assert np.linalg.norm(x - np.linalg.solve(Z + ZF, b)) / np.linalg.norm(x) < 1e-11


def test_pipeline_against_dense_efie(sphere480):
    import efie_problem as ep
    P = sphere480
    Z = ep.EntryEvaluator(P.rwg).dense()
    Zs = np.triu(Z) + np.triu(Z, 1).T
    b = P.plane_wave([0, 0, -1], [1, 0, 0])
    nl = len(P.leaf_ptr) - 1
    F = schur.setup(P, ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist()))), 0.0)
    x, it, rr, ok = krylov.solve(krylov.System(P, F), b, tol=1e-10, restart=30)
    xd = np.linalg.solve(Zs, b)
    assert ok and np.linalg.norm(x - xd) / np.linalg.norm(xd) < 10 * 1e-3


# ---- ordering (Algorithm 1 with RCM) --------------------------------------------------------
def test_rcm_path_and_grid():
    n = 20
    path = [(i, i + 1) for i in range(n - 1)]
    o = ordering.rcm(n, path)
    assert sorted(o.tolist()) == list(range(n)) and ordering.bandwidth(n, path, o) == 1
    w = 6
    grid = [(r * w + c, r * w + c + 1) for r in range(w) for c in range(w - 1)] + \
           [(r * w + c, (r + 1) * w + c) for r in range(w - 1) for c in range(w)]
    rng = np.random.default_rng(1)
    relabel = rng.permutation(w * w)
    g2 = [(int(relabel[a]), int(relabel[b])) for a, b in grid]
    o = ordering.rcm(w * w, g2)
    assert ordering.bandwidth(w * w, g2, o) <= w
    assert ordering.bandwidth(w * w, g2, o) < ordering.bandwidth(w * w, g2)


def test_rcm_on_sphere_graph_vs_scipy(sphere1920):
    P = sphere1920
    nl = len(P.leaf_ptr) - 1
    pairs = list(zip(P.near_t.tolist(), P.near_s.tolist()))
    o = ordering.rcm(nl, pairs)
    assert sorted(o.tolist()) == list(range(nl))
    bw = ordering.bandwidth(nl, pairs, o)
    assert bw <= ordering.bandwidth(nl, pairs)
    r = [t for t, s in pairs] + [s for t, s in pairs]
    c = [s for t, s in pairs] + [t for t, s in pairs]
    A = ssp.csr_matrix((np.ones(len(r)), (r, c)), shape=(nl, nl))
    bs = ordering.bandwidth(nl, pairs, csg.reverse_cuthill_mckee(A, symmetric_mode=True))
    assert bw <= 1.1 * bs + 1


def test_rcm_disconnected_components():
    pairs = [(0, 3), (3, 5), (1, 2), (4, 4)]
    o = ordering.rcm(6, pairs)
    assert sorted(o.tolist()) == list(range(6))


def test_rcm_start_rule_hand_traced():
    """A path 1-2-3-4-5-6-7 with node 0 hanging on 4.  The search starts at the minimum-
    (degree, index) node 0 (5 levels), moves to 1 (7 levels), and stops (7 is no deeper):
    Cuthill-McKee from 1 is 1 2 3 4 0 5 6 7 (0 before 5: lower degree), reversed."""
    pairs = [(1, 2), (2, 3), (3, 4), (4, 5), (5, 6), (6, 7), (0, 4)]
    assert ordering.rcm(8, pairs).tolist() == [7, 6, 5, 0, 4, 3, 2, 1]


# ---- Sloan's ordering (the best ordering of Sec. 3.3, Tables 3-4) ------------------------------
def test_sloan_path_runs_end_to_end():
    rng = np.random.default_rng(0)
    perm = rng.permutation(10)
    pairs = [(int(perm[i]), int(perm[i + 1])) for i in range(9)]
    o = ordering.sloan(10, pairs)
    # from the lower-index end of the path to the other end
    assert o.tolist() == (perm[::-1] if perm[-1] < perm[0] else perm).tolist()


def test_sloan_hand_traced():
    """Edges 3-0, 0-4, 4-1, 0-1, 1-2.  Start 2 (degree 1, lowest index), end 3; distances to
    3: 2->3, 1->2, 4->2, 0->1, 3->0; P = 2 dist - (deg + 1) = {2: 4, 1: 0, 4: 1, 0: -2, 3: -2}.
    Number 2 (1 -> 1, preactive; then active: 2, its neighbours 0 -> -1, 4 -> 2); the tie 1/4 at
    2 goes to 1 (active: 0 -> 0 then 3 -> -1 and 4 -> 3 via 0, 4 -> 4 and 0 -> 1 via 4); then 4
    (priority 4), 0 (1), 3."""
    assert ordering.sloan(5, [(3, 0), (0, 4), (4, 1), (0, 1), (1, 2)]).tolist() == [2, 1, 4, 0, 3]
    assert ordering.sloan(5, [(0, 1), (1, 2), (2, 3), (1, 3), (3, 4)]).tolist() == [0, 1, 2, 3, 4]


def _grid(a, b, seed):
    idx = lambda i, j: i * b + j
    pr = []
    for i in range(a):
        for j in range(b):
            if i + 1 < a:
                pr.append((idx(i, j), idx(i + 1, j)))
            if j + 1 < b:
                pr.append((idx(i, j), idx(i, j + 1)))
            if i + 1 < a and j + 1 < b:
                pr.append((idx(i, j), idx(i + 1, j + 1)))
    p = np.random.default_rng(seed).permutation(a * b)
    return a * b, [(int(p[x]), int(p[y])) for x, y in pr]


def test_sloan_profile_not_above_rcm_on_grids():
    """Profile reduction is what Sloan's algorithm is for: on triangulated grids (the meshes of
    the plate workloads) its profile is at most RCM's and far below a random numbering's."""
    for a, b in ((5, 20), (10, 30), (17, 17)):
        n, pairs = _grid(a, b, a)
        o = ordering.sloan(n, pairs)
        assert sorted(o.tolist()) == list(range(n))
        ps = ordering.profile(n, pairs, o)
        assert ps <= ordering.profile(n, pairs, ordering.rcm(n, pairs))
        assert ps < 0.2 * ordering.profile(n, pairs)


def test_sloan_disconnected_components():
    pairs = [(0, 3), (3, 5), (1, 2), (4, 4)]
    o = ordering.sloan(6, pairs)
    assert sorted(o.tolist()) == list(range(6))
    assert o.tolist()[:3] == [0, 3, 5]      # component of node 0 first, then {1, 2}, then {4}
    assert o.tolist()[3:] == [1, 2, 4]


# ---- block-Jacobi comparison preconditioner (Sec. 1: the block diagonal preconditioner) --------
def test_block_jacobi_operator_is_dense_M_inverse_Z():
    """M^{-1} (Z_N + Z_F) with M = the near-field diagonal blocks, against its dense form."""
    rng = np.random.default_rng(21)
    sizes = [3, 5, 4, 2, 6]
    pairs = [(0, 0), (0, 1), (1, 1), (1, 2), (2, 2), (2, 3), (3, 3), (3, 4), (4, 4)]
    far = [((0, 2), 0.3 * (rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))))]
    p, Z, ZF = block_problem(sizes, pairs, rng, far=far)
    order = np.array([2, 0, 4, 1, 3])
    S = krylov.BlockJacobi(p, order)
    lp = p.leaf_ptr
    Mdense = np.zeros_like(Z)
    for t in range(5):
        Mdense[lp[t]:lp[t + 1], lp[t]:lp[t + 1]] = Z[lp[t]:lp[t + 1], lp[t]:lp[t + 1]]
    x = rng.standard_normal(Z.shape[0]) + 1j * rng.standard_normal(Z.shape[0])
    y = S.apply_A(S.to_new(x))                       # in the block order
    ref = np.linalg.solve(Mdense, (Z + ZF) @ x)      # in the original order
    assert np.linalg.norm(S.to_orig(y) - ref) / np.linalg.norm(ref) < 1e-12
    b = rng.standard_normal(Z.shape[0]) + 1j * rng.standard_normal(Z.shape[0])
    xs, it, rr, ok = krylov.solve(S, b, tol=1e-13, restart=30)
    assert ok and np.linalg.norm(xs - np.linalg.solve(Z + ZF, b)) / np.linalg.norm(xs) < 1e-11


def test_block_jacobi_exact_on_block_diagonal_systems():
    """No off-diagonal near blocks and no far field: M = Z, so one Arnoldi step."""
    rng = np.random.default_rng(22)
    sizes = [4, 3, 5]
    p, Z, ZF = block_problem(sizes, [(0, 0), (1, 1), (2, 2)], rng)
    S = krylov.BlockJacobi(p, np.array([1, 2, 0]))
    b = rng.standard_normal(Z.shape[0]) + 1j * rng.standard_normal(Z.shape[0])
    x, it, rr, ok = krylov.solve(S, b, tol=1e-12, restart=10)
    assert ok and it == 1
    assert np.linalg.norm(x - np.linalg.solve(Z, b)) / np.linalg.norm(x) < 1e-12


def test_preconditioned_spectrum_clusters_near_one(sphere480):
    """Fig. 13's observation, as a soft check on the 480-unknown sphere: the eigenvalues of the
    Eq. 28 operator A = D^{-1} [D + L^{-1} Z_F L^{-T}] lie closer to 1 than those of Z scaled by
    its own diagonal, and A is exactly the identity when the far field is left out (Eq. 21)."""
    P = sphere480
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    S = krylov.System(P, schur.setup(P, order, fill_tol=0.0))
    n = S.n
    I = np.eye(n, dtype=np.complex128)
    A = np.stack([S.apply_A(I[:, j]) for j in range(n)], axis=1)
    Z = np.stack([S.Z_orig(I[:, j]) for j in range(n)], axis=1)
    lam_a = np.linalg.eigvals(A)
    lam_z = np.linalg.eigvals(Z / np.diag(Z)[:, None])
    da, dz = np.abs(lam_a - 1.0), np.abs(lam_z - 1.0)
    assert np.median(da) < 0.5 * np.median(dz) and np.max(da) < np.max(dz)
    # without Z_F the operator is D^{-1} D = I
    N = np.stack([S.D_solve(S.D_mul(I[:, j])) for j in range(n)], axis=1)
    assert np.abs(N - I).max() < 1e-10


# ---- null-field comparison preconditioner (Sec. 3: one-sided near-field scaling without fill) ----
def _cycle(rng, far=None):
    """Five blocks on a cycle 0-1-2-3-4-0: eliminating block 0 couples 1 and 4, which are not
    near-field neighbours, so the complete elimination fills (1, 4) and later pairs."""
    sizes = [3, 5, 4, 2, 6]
    pairs = [(t, t) for t in range(5)] + [(0, 1), (1, 2), (2, 3), (3, 4), (0, 4)]
    return block_problem(sizes, pairs, rng, far=far, diag_boost=6.0)


def _near_block_mask(F, near_pairs):
    off = np.concatenate([[0], np.cumsum(F.size)])
    n = int(off[-1])
    mask = np.zeros((n, n), dtype=bool)
    for i in range(F.nb):
        for j in range(F.nb):
            if i == j or (max(i, j), min(i, j)) in near_pairs:
                mask[off[i]:off[i + 1], off[j]:off[j + 1]] = True
    return mask


def test_null_field_factor_is_the_incomplete_factorisation_of_the_near_pattern():
    """The elimination without fill is characterised without reference to its algorithm: L is
    unit lower triangular with blocks only on near-field pairs, D is block diagonal, and
    M = L D L^T equals Z_N on every near-field block pair (these equations have one solution).
    Off the pattern M differs from Z_N, which the complete factorisation reproduces exactly."""
    rng = np.random.default_rng(41)
    p, Z, ZF = _cycle(rng)
    for order in (np.arange(5), np.array([2, 0, 4, 1, 3])):
        S = krylov.NullField(p, order)
        F = S.F
        assert F.S == schur.near_lists(5, list(F.near_pairs))
        Zn = Z[np.ix_(S.new2orig, S.new2orig)]
        L, D = schur.ldlt_dense(F)
        mask = _near_block_mask(F, F.near_pairs)
        assert np.all(L[~mask] == 0) and np.allclose(np.diag(L), 1) and np.all(np.triu(L, 1) == 0)
        M = L @ D @ L.T
        assert np.abs(M - Zn)[mask].max() < 1e-12 * np.abs(Zn).max()
        assert np.abs(M - Zn)[~mask].max() > 1e-3 * np.abs(Zn).max()
        Fc = schur.setup(p, order, fill_tol=0.0)
        Lc, Dc = schur.ldlt_dense(Fc)
        assert np.abs(Lc @ Dc @ Lc.T - Zn).max() < 1e-12 * np.abs(Zn).max()


def test_null_field_on_the_sphere_reproduces_the_near_field_on_its_pattern(sphere480):
    """The same characterisation on the 480-unknown EFIE sphere in RCM order, where the complete
    elimination fills: L has no block outside the near-field pattern, L D L^T equals Z_N on
    every near-field block pair, and differs from it off the pattern (the dropped fill)."""
    P = sphere480
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    S = krylov.NullField(P, order)
    F = S.F
    assert sum(len(x) for x in F.S) < sum(len(x) for x in schur.symbolic_fill(nl, list(F.near_pairs)))
    n = S.n
    Zn = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        u = np.zeros(n, dtype=np.complex128)
        u[S.new2cl] = e
        Zn[:, j] = S.near_cluster(u)[S.new2cl]
    L, D = schur.ldlt_dense(F)
    mask = _near_block_mask(F, F.near_pairs)
    assert np.all(L[~mask] == 0)
    M = L @ D @ L.T
    scale = np.abs(Zn).max()
    assert np.abs(M - Zn)[mask].max() < 1e-11 * scale
    assert np.abs(M - Zn)[~mask].max() > 1e-6 * scale


def test_null_field_equals_the_schur_factor_when_the_pattern_has_no_fill():
    """A block-tridiagonal near field in its natural order has no fill-in: the two
    eliminations coincide, M = Z_N, so with no far field GMRES ends after one step."""
    rng = np.random.default_rng(42)
    sizes = [4, 3, 5, 2]
    pairs = [(t, t) for t in range(4)] + [(0, 1), (1, 2), (2, 3)]
    p, Z, ZF = block_problem(sizes, pairs, rng, diag_boost=6.0)
    order = np.arange(4)
    S = krylov.NullField(p, order)
    Fc = schur.setup(p, order, fill_tol=0.0)
    assert S.F.S == Fc.S
    for k in range(4):
        assert np.array_equal(S.F.D[k], Fc.D[k])
    for key in Fc.W:
        assert np.array_equal(S.F.W[key], Fc.W[key])
    b = rng.standard_normal(Z.shape[0]) + 1j * rng.standard_normal(Z.shape[0])
    x, it, rr, ok = krylov.solve(S, b, tol=1e-12, restart=10)
    assert ok and it == 1
    assert np.linalg.norm(x - np.linalg.solve(Z, b)) / np.linalg.norm(x) < 1e-12


def test_null_field_operator_is_dense_M_inverse_Z_and_solves():
    """M^{-1} (Z_N + Z_F) against a dense solve with the (pinned) M, and a tight solve of the
    full system."""
    rng = np.random.default_rng(43)
    far = [((1, 3), 0.3 * (rng.standard_normal((5, 2)) + 1j * rng.standard_normal((5, 2))))]
    p, Z, ZF = _cycle(rng, far=far)
    order = np.array([2, 0, 4, 1, 3])
    S = krylov.NullField(p, order)
    L, D = schur.ldlt_dense(S.F)
    P = np.eye(Z.shape[0])[S.new2orig]            # P x_orig = x_new
    M = P.T @ (L @ D @ L.T) @ P                   # M in the original order
    x = rng.standard_normal(Z.shape[0]) + 1j * rng.standard_normal(Z.shape[0])
    ref = np.linalg.solve(M, (Z + ZF) @ x)
    assert np.linalg.norm(S.to_orig(S.apply_A(S.to_new(x))) - ref) / np.linalg.norm(ref) < 1e-12
    b = rng.standard_normal(Z.shape[0]) + 1j * rng.standard_normal(Z.shape[0])
    assert np.linalg.norm(S.rhs(b) - S.to_new(np.linalg.solve(M, b))) < 1e-12 * np.linalg.norm(b)
    xs, it, rr, ok = krylov.solve(S, b, tol=1e-13, restart=30)
    assert ok and np.linalg.norm(xs - np.linalg.solve(Z + ZF, b)) / np.linalg.norm(xs) < 1e-11


# ---- Sec. 3.4 read as compression during the setup (the abstract's reading) ---------------------
def test_compression_in_setup_changes_exactly_the_later_updates():
    """Star 0-1, 0-2: eliminating block 0 couples 1 and 2, so W_12 is a fill-in block.  With
    the compression during setup, W_12 is truncated before the update of step 1 uses it:
    D_0, D_1, W_01, W_02 equal the post-factorisation reading's, and
    D_2(setup) - D_2(after) = A_21 (W_12 - trunc(W_12)), with A_21 = D_1 W_12 (the symmetric
    update's left factor), bounded by ||A_21|| fill_tol ||W_12||."""
    rng = np.random.default_rng(31)
    sizes = [4, 6, 5]
    p, Z, ZF = block_problem(sizes, [(0, 0), (0, 1), (0, 2), (1, 1), (2, 2)], rng, diag_boost=6.0)
    order = np.array([0, 1, 2])
    tol = 0.3
    Fa = schur.setup(p, order, fill_tol=tol)
    Fb = schur.setup(p, order, fill_tol=tol, compress_in_setup=True)
    assert Fa.S[1] == [2] and (2, 1) not in Fa.near_pairs           # W_12 is a fill-in block
    for k in (0, 1):
        assert np.allclose(Fa.D[k], Fb.D[k], rtol=0, atol=1e-13)
    for key in ((0, 1), (0, 2)):
        assert np.array_equal(Fa.W[key], Fb.W[key])
    W12 = Fa.W[(1, 2)]
    T12, r = schur.compress_block(W12, tol)
    assert 0 <= r < min(W12.shape)                                   # the truncation bites
    assert np.allclose(Fb.W[(1, 2)], T12, rtol=0, atol=1e-13)
    A21 = Fa.D[1] @ W12
    dD = Fb.D[2] - Fa.D[2]
    assert np.linalg.norm(dD - (A21.T @ (W12 - T12))) <= 1e-12 * np.linalg.norm(dD)
    assert np.linalg.norm(dD) <= np.linalg.norm(A21) * tol * np.linalg.norm(W12) * 1.0001


def test_compression_in_setup_zero_tolerance_is_exact(sphere480):
    P = sphere480
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    Fa = schur.setup(P, order, fill_tol=0.0)
    Fb = schur.setup(P, order, fill_tol=0.0, compress_in_setup=True)
    for k in range(Fa.nb):
        assert np.array_equal(Fa.D[k], Fb.D[k])
