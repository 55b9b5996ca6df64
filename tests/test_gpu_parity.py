"""GPU-vs-oracle parity through the C-ABI (libhmsolve.so) on seeded problems.

Tolerances: FP64 throughout.  Factor blocks and single operator applications agree to
1e-10 relative (explicit inverses vs LU solves, different summation order); solutions
of the full preconditioned GMRES to 1e-8 relative 2-norm with iteration counts within
+-1 (the GPU orthogonalises by CGS2, the oracle by MGS: same Krylov space up to rounding).
"""
import numpy as np
import pytest
import torch

import paper_2111_13483_gb300 as hm
from oracle import krylov, ordering, schur
from refs import truncated_at

pytestmark = pytest.mark.gpu


def oracle_factor(P, fill_tol=0.0):
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    F = schur.setup(P, order, fill_tol=fill_tol)
    return order, F, krylov.System(P, F)


@pytest.fixture(scope="module")
def small(sphere480):
    P = sphere480
    order, F, S = oracle_factor(P)
    h = hm.hmat_create(P, ordering=1, fill_tol=0.0)
    hm.precond_setup(h)
    return P, order, F, S, h


@pytest.fixture(scope="module")
def cfg1(sphere1920):
    P = sphere1920
    order, F, S = oracle_factor(P)
    h = hm.hmat_create(P, ordering=1, fill_tol=0.0)
    hm.precond_setup(h)
    return P, order, F, S, h


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.mark.parametrize("which", ["small", "cfg1"])
def test_order_and_fill_match_oracle(which, request):
    P, order, F, S, h = request.getfixturevalue(which)
    assert np.array_equal(hm.hm_get_order(h), order)
    ptr, idx = hm.hm_get_fill(h)
    for k in range(F.nb):
        assert list(idx[ptr[k]:ptr[k + 1]]) == F.S[k]
    assert np.array_equal(hm.hm_get_index_map(h), S.new2orig)


@pytest.mark.parametrize("which", ["small", "cfg1"])
def test_factor_blocks_match_oracle(which, request):
    P, order, F, S, h = request.getfixturevalue(which)
    for k in range(F.nb):
        nk = int(F.size[k])
        D = hm.hm_get_block(h, 0, k, (nk, nk))
        assert rel(D, F.D[k]) < 1e-10, k
        Di = hm.hm_get_block(h, 1, k, (nk, nk))
        assert rel(Di, np.linalg.inv(F.D[k])) < 1e-9, k
        if F.S[k]:
            M = int(sum(F.size[j] for j in F.S[k]))
            Wk = hm.hm_get_block(h, 2, k, (nk, M))
            Wo = np.concatenate([F.W[(k, j)] for j in F.S[k]], axis=1)
            assert rel(Wk, Wo) < 1e-10, k


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x.T)).cuda()


def _host(t):
    return t.cpu().numpy().T


@pytest.mark.parametrize("which", ["small", "cfg1"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_operators_match_oracle(which, nrhs, request):
    P, order, F, S, h = request.getfixturevalue(which)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((S.n, nrhs)) + 1j * rng.standard_normal((S.n, nrhs))
    dx = _dev(X)
    dy = torch.empty_like(dx)
    refs = {hm.hmsolve.OP_A: S.apply_A, hm.hmsolve.OP_LINV: S.L_inv, hm.hmsolve.OP_LTINV: S.LT_inv,
            hm.hmsolve.OP_ZF: S.far_new, hm.hmsolve.OP_DINV: S.D_solve, hm.hmsolve.OP_Z: S.Z_orig}
    for op, f in refs.items():
        hm.hm_apply(h, op, dx, dy)
        torch.cuda.synchronize()
        Y = _host(dy)
        for c in range(nrhs):
            assert rel(Y[:, c], f(X[:, c])) < 1e-10, (op, c)


@pytest.mark.parametrize("which", ["small", "cfg1"])
def test_solve_matches_oracle(which, request):
    P, order, F, S, h = request.getfixturevalue(which)
    b = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    x, it, rr, code = hm.solve(h, b, tol=1e-4, restart=30, maxit=2000)
    xo, ito, rro, ok = krylov.solve(S, b, tol=1e-4, restart=30)
    assert code == 0 and ok
    assert abs(int(it[0]) - ito) <= 1
    assert rel(x, xo) <= 1e-8
    assert rr[0] <= 1e-4


def test_solve_tight_tolerance_and_restarts(cfg1):
    P, order, F, S, h = cfg1
    b = P.plane_wave([1.0, 0.0, 0.0], [0.0, 0.0, 1.0])
    x, it, rr, code = hm.solve(h, b, tol=1e-10, restart=5, maxit=2000)
    xo, ito, rro, ok = krylov.solve(S, b, tol=1e-10, restart=5)
    assert code == 0 and ok and abs(int(it[0]) - ito) <= 1
    assert rel(x, xo) <= 1e-8


def test_multi_rhs_equals_single(cfg1):
    P, order, F, S, h = cfg1
    rng = np.random.default_rng(3)
    B = np.stack([P.plane_wave([np.cos(p), np.sin(p), 0.0], [0.0, 0.0, 1.0]) for p in rng.uniform(0, 6.28, 5)], 1)
    X, its, rrs, code = hm.solve(h, B, tol=1e-6, restart=30)
    assert code == 0
    for c in range(B.shape[1]):
        x1, it1, rr1, c1 = hm.solve(h, B[:, c], tol=1e-6, restart=30)
        assert it1[0] == its[c]
        assert np.array_equal(x1, X[:, c]), c          # batch invariant: bitwise


def test_solve_device_matches_host(cfg1):
    P, order, F, S, h = cfg1
    b = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    x, it, rr, code = hm.solve(h, b, tol=1e-6)
    dV = torch.from_numpy(b[None, :].copy()).cuda()
    dI = torch.zeros_like(dV)
    it2, rr2, code2 = hm.solve_device(h, dV, dI, tol=1e-6)
    assert code2 == 0 and it2[0] == it[0]
    assert np.array_equal(dI.cpu().numpy()[0], x)


def test_true_residual_small(cfg1):
    P, order, F, S, h = cfg1
    b = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    x, it, rr, code = hm.solve(h, b, tol=1e-8)
    assert np.linalg.norm(b - S.Z_orig(x)) / np.linalg.norm(b) < 1e-6


# ---- mixed precision: complex-FP32 operator inside FP64 refinement ----------------------
@pytest.fixture(scope="module")
def cfg1_mixed(sphere1920):
    h = hm.hmat_create(sphere1920, ordering=1, fill_tol=0.0, precision=1)
    hm.precond_setup(h)
    return h


@pytest.fixture(scope="module")
def cfg1_tight(cfg1):
    """The oracle's solve of the same discrete system at tolerance 1e-10 (per column)."""
    P, order, F, S, h = cfg1
    B = np.stack([P.plane_wave([-np.cos(p), -np.sin(p), 0.0], [0.0, 0.0, -1.0])
                  for p in (0.0, 1.3, 2.9)], axis=1)
    X = np.stack([krylov.solve(S, B[:, c], tol=1e-10, restart=30)[0] for c in range(B.shape[1])], axis=1)
    return B, X


def test_mixed_factors_close_to_fp64(cfg1, cfg1_mixed):
    """FP32 Schur products, FP64 pivots: the factors stay within FP32 rounding of the oracle."""
    P, order, F, S, h = cfg1
    for k in range(0, F.nb, 5):
        nk = int(F.size[k])
        D = hm.hm_get_block(cfg1_mixed, 0, k, (nk, nk))
        assert rel(D, F.D[k]) < 1e-4, k


def test_update_schedules_match(cfg1, sphere1920):
    """The complex-FP32 Schur updates on the CUDA cores (kind 1) and on the tensor cores (kind 2,
    3xTF32): every D_k, D_k^{-1} and panel W_k within FP32 rounding of the oracle's FP64 factors
    and of each other, and each kind's setup bitwise reproducible."""
    P, order, F, S, h = cfg1
    got = {}
    for kind in (1, 2, 2):
        g = hm.hmat_create(sphere1920, ordering=1, precision=1)
        hm.hmsolve.hm_set_update_schedule(g, kind)
        hm.precond_setup(g)
        blocks = []
        for k in range(F.nb):
            nk = int(F.size[k])
            D = hm.hm_get_block(g, 0, k, (nk, nk))
            assert rel(D, F.D[k]) < 1e-4, (kind, k)
            blocks.append(D)
            if F.S[k]:
                M = int(sum(F.size[j] for j in F.S[k]))
                Wk = hm.hm_get_block(g, 2, k, (nk, M))
                Wo = np.concatenate([F.W[(k, j)] for j in F.S[k]], axis=1)
                assert rel(Wk, Wo) < 1e-3, (kind, k)
                blocks.append(Wk)
        if kind in got:
            assert all(np.array_equal(x, y) for x, y in zip(blocks, got[kind]))
        got[kind] = blocks
        hm.hmat_destroy(g)
    assert max(rel(x, y) for x, y in zip(got[1], got[2])) < 1e-3


@pytest.mark.parametrize("prec", [0, 1])
def test_pivot_schedules_bitwise_equal(sphere1920, prec):
    """The pivot inverses on clusters of 2, 4 and 8 CTAs do each entry's Gauss-Jordan operations
    of the one-CTA kernel: D_k^{-1}, the panels built from them and a solve are bitwise those of
    one CTA (FP64 and mixed setups), and within 1e-9 of the oracle's inverses (FP64)."""
    nl = len(sphere1920.leaf_ptr) - 1
    F = schur.setup(sphere1920, ordering.rcm(nl, list(zip(sphere1920.near_t.tolist(), sphere1920.near_s.tolist()))),
                    fill_tol=0.0) if prec == 0 else None
    b = sphere1920.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    ref = None
    for ctas in (1, 2, 4, 8):
        g = hm.hmat_create(sphere1920, ordering=1, precision=prec, fill_tol=1e-2)
        hm.hmsolve.hm_set_pivot_schedule(g, ctas)
        hm.precond_setup(g)
        ptr, idx = hm.hm_get_fill(g)
        size = np.diff(sphere1920.leaf_ptr)[hm.hm_get_order(g)]
        got = []
        for k in range(len(size)):
            nk = int(size[k])
            Di = hm.hm_get_block(g, 1, k, (nk, nk))
            if F is not None and k % 7 == 0:
                assert rel(Di, np.linalg.inv(F.D[k])) < 1e-9, (ctas, k)
            got.append(Di)
            if ptr[k + 1] > ptr[k]:
                got.append(hm.hm_get_block(g, 2, k, (nk, int(size[idx[ptr[k]:ptr[k + 1]]].sum()))))
        x, it, rr, code = hm.solve(g, b, tol=1e-5, restart=30)
        got.append(x)
        if ref is None:
            ref = got
        else:
            assert all(np.array_equal(u, v) for u, v in zip(got, ref)), ctas
        hm.hmat_destroy(g)
    with pytest.raises(hm.HMError):
        hm.hmsolve.hm_set_pivot_schedule(hm.hmat_create(sphere1920, ordering=1), 3)


def test_mixed_solution_error_against_tight_oracle(cfg1, cfg1_mixed, cfg1_tight):
    """The FP64 refinement loop stops on the true residual ||V - Z I||/||V||; at 1e-5 (the
    setting the benchmark uses for its 1e-4 error bar) the solution is within 1e-4 of the
    oracle's tight solve, and the residual is verified with the oracle's own H-matrix
    product."""
    P, order, F, S, h = cfg1
    B, X = cfg1_tight
    I, its, rr, code = hm.solve(cfg1_mixed, B, tol=1e-5, restart=30)
    assert code == 0
    for c in range(B.shape[1]):
        assert rr[c] <= 1e-5
        assert np.linalg.norm(B[:, c] - S.Z_orig(I[:, c])) / np.linalg.norm(B[:, c]) <= 1.01e-5
        assert rel(I[:, c], X[:, c]) <= 1e-4


def test_mixed_multi_rhs_equals_single(cfg1_mixed, cfg1_tight):
    B, X = cfg1_tight
    I, its, rr, code = hm.solve(cfg1_mixed, B, tol=1e-5, restart=30)
    assert code == 0
    for c in range(B.shape[1]):
        x1, it1, rr1, c1 = hm.solve(cfg1_mixed, B[:, c], tol=1e-5, restart=30)
        assert it1[0] == its[c] and np.array_equal(x1, I[:, c]), c


# ---- Sec. 3.4 fill-in compression ------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg1_compressed(sphere1920):
    P = sphere1920
    order, F, S = oracle_factor(P, fill_tol=1e-2)
    h = hm.hmat_create(P, ordering=1, fill_tol=1e-2)
    hm.precond_setup(h)
    return P, order, F, S, h


def test_compression_ranks_and_blocks_match_oracle(cfg1_compressed):
    """Ranks equal the oracle's truncated-SVD ranks (the same Frobenius-tail rule), and the
    compressed coefficient blocks equal the oracle's truncations."""
    P, order, F, S, h = cfg1_compressed
    ptr, idx = hm.hm_get_fill(h)
    ranks = hm.hmsolve.hm_get_fill_ranks(h)
    n_comp = 0
    for k in range(F.nb):
        for a, j in enumerate(F.S[k]):
            r_gpu = int(ranks[ptr[k] + a])
            r_ora = F.rank.get((k, j), -1)
            assert r_gpu == r_ora, (k, j, r_gpu, r_ora)
            n_comp += r_gpu >= 0
        if F.S[k]:
            nk = int(F.size[k])
            M = int(sum(F.size[j] for j in F.S[k]))
            Wk = hm.hm_get_block(h, 2, k, (nk, M))
            Wo = np.concatenate([F.Wc[(k, j)] for j in F.S[k]], axis=1)
            assert rel(Wk, Wo) < 1e-8, k
    assert n_comp > 0
    st = hm.hmat_stats(h)
    assert st["coef_entries"] < st["coef_entries_dense"]


@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_compressed_operators_match_oracle(cfg1_compressed, nrhs):
    """Compressed fill-in blocks are stored as their factors (U_r Sigma_r, V_r) and applied as
    two products; the oracle applies the expanded truncations: equal up to rounding.  The
    store holds exactly the oracle's Table 6 count of coefficient entries."""
    P, order, F, S, h = cfg1_compressed
    st = hm.hmat_stats(h)
    assert st["coef_entries"] == schur.nnz_coefficients(F) - int(np.sum(F.size))
    rng = np.random.default_rng(17 + nrhs)
    X = rng.standard_normal((S.n, nrhs)) + 1j * rng.standard_normal((S.n, nrhs))
    dx = _dev(X)
    for op, f in ((hm.hmsolve.OP_LINV, S.L_inv), (hm.hmsolve.OP_LTINV, S.LT_inv), (hm.hmsolve.OP_A, S.apply_A)):
        dy = torch.empty_like(dx)
        hm.hm_apply(h, op, dx, dy)
        Y = _host(dy)
        for c in range(nrhs):
            assert rel(Y[:, c], f(X[:, c])) < 1e-10, (op, c)


def test_compressed_mixed_operators_and_solve(cfg1_compressed, sphere1920):
    P, order, F, S, h64 = cfg1_compressed
    h = hm.hmat_create(sphere1920, ordering=1, fill_tol=1e-2, precision=1)
    hm.precond_setup(h)
    ranks32 = hm.hmsolve.hm_get_fill_ranks(h)
    ranks64 = hm.hmsolve.hm_get_fill_ranks(h64)
    assert np.mean(ranks32 == ranks64) > 0.95
    Wm = truncated_at(F, h)
    rng = np.random.default_rng(19)
    X = rng.standard_normal((S.n, 5)) + 1j * rng.standard_normal((S.n, 5))
    refs = ((hm.hmsolve.OP_LINV, lambda x: S.join(schur.sweep_forward(F, S.split(x), W=Wm))),
            (hm.hmsolve.OP_LTINV, lambda x: S.join(schur.sweep_backward(F, S.split(x), W=Wm))))
    for op, f in refs:
        dy = torch.empty_like(_dev(X))
        hm.hm_apply(h, hm.hmsolve.OP32 + op, _dev(X), dy)
        Y = _host(dy)
        for c in range(5):
            assert rel(Y[:, c], f(X[:, c])) < 1e-4, (op, c)
    b = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    x, it, rr, code = hm.solve(h, b, tol=1e-5, restart=30)
    assert code == 0
    assert np.linalg.norm(b - S.Z_orig(x)) / np.linalg.norm(b) <= 1.01e-5


def test_compressed_solve_matches_oracle(cfg1_compressed):
    P, order, F, S, h = cfg1_compressed
    b = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    x, it, rr, code = hm.solve(h, b, tol=1e-6, restart=30)
    xo, ito, rro, ok = krylov.solve(S, b, tol=1e-6, restart=30)
    assert code == 0 and ok and abs(int(it[0]) - ito) <= 1
    assert rel(x, xo) <= 1e-8


# ---- sweep schedules: (groups, kind) choices that give bitwise the same sweeps ------------------
# kind 1: one block row per CTA, 2: two-row super-rows, 3: chain CTA + helpers (CUDA cores,
# the same summation order), 5 / 6: one block row per CTA in clusters of 8 / 16 CTAs that read
# their in-cluster dependencies through distributed shared memory (complex FP32; the same
# summation order; FP64 sweeps take kind 1 for them); kind 4: complex FP32 on the tensor cores
# (its own fixed order, bitwise the same for every column grouping; FP64 sweeps take kind 1)
@pytest.mark.parametrize("prec", [0, 1])
def test_sweep_schedules_bitwise_equal(cfg1, cfg1_mixed, prec):
    P, order, F, S, h64 = cfg1
    h = h64 if prec == 0 else cfg1_mixed
    ops = (hm.hmsolve.OP_LINV, hm.hmsolve.OP_LTINV, hm.hmsolve.OP_A)
    if prec == 1:
        ops = tuple(hm.hmsolve.OP32 + o for o in ops)
    families = [[(g, k, 0) for g in (1, 2, 4) for k in (1, 2, 3, 5, 6)] + [(g, 1, t) for g in (1, 2, 4) for t in (1, 2)]]
    tc = [(g, 4, 0) for g in (1, 2, 4)]
    if prec == 0:
        families[0] += tc
    else:
        families.append(tc)
    rng = np.random.default_rng(11)
    for nrhs in (1, 5, 16, 64):
        X = rng.standard_normal((S.n, nrhs)) + 1j * rng.standard_normal((S.n, nrhs))
        dx = _dev(X)
        refs = []
        for fam in families:
            ref = {}
            for sched in fam:
                hm.hmsolve.hm_set_sweep_schedule(h, *sched)
                for op in ops:
                    dy = torch.empty_like(dx)
                    hm.hm_apply(h, op, dx, dy)
                    torch.cuda.synchronize()
                    Y = _host(dy)
                    if op not in ref:
                        ref[op] = Y
                        if prec == 0 and op == hm.hmsolve.OP_LINV:
                            for c in range(nrhs):
                                assert rel(Y[:, c], S.L_inv(X[:, c])) < 1e-10
                    else:
                        assert np.array_equal(Y, ref[op]), (sched, op, nrhs)
            refs.append(ref)
        if len(refs) == 2:   # tensor cores (3xTF32) against CUDA cores (FP32): FP32-level agreement
            for op in ops:
                for c in range(nrhs):
                    assert rel(refs[1][op][:, c], refs[0][op][:, c]) < 1e-5, (op, c)
        hm.hmsolve.hm_set_sweep_schedule(h, 0, 0)


# ---- plate (the GMRES(50) workload's geometry, 2 x 2 lambda on the same grid) ------------------
@pytest.fixture(scope="module")
def plate_cfg():
    import efie_problem as ep
    P = ep.build("plate1160")
    order, F, S = oracle_factor(P)
    return P, order, F, S


@pytest.mark.parametrize("prec", [0, 1])
def test_plate_solve_matches_oracle(plate_cfg, prec):
    P, order, F, S = plate_cfg
    h = hm.hmat_create(P, ordering=1, fill_tol=0.0, precision=prec)
    hm.precond_setup(h)
    assert np.array_equal(hm.hm_get_order(h), order)
    # normal and oblique incidence, both with a field component tangential to the plate
    B = np.stack([P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0]),
                  P.plane_wave([0.6, 0.0, -0.8], [0.8, 0.0, 0.6])], axis=1)
    assert np.all(np.linalg.norm(B, axis=0) > 0)
    if prec == 0:
        X, its, rr, code = hm.solve(h, B, tol=1e-6, restart=50)
        assert code == 0
        for c in range(B.shape[1]):
            xo, ito, rro, ok = krylov.solve(S, B[:, c], tol=1e-6, restart=50)
            assert ok and abs(int(its[c]) - ito) <= 1
            assert rel(X[:, c], xo) <= 1e-8
    else:
        X, its, rr, code = hm.solve(h, B, tol=1e-5, restart=50)
        assert code == 0
        for c in range(B.shape[1]):
            xt = krylov.solve(S, B[:, c], tol=1e-10, restart=50)[0]
            assert np.linalg.norm(B[:, c] - S.Z_orig(X[:, c])) / np.linalg.norm(B[:, c]) <= 1.01e-5
            assert rel(X[:, c], xt) <= 1e-4


# ---- Sloan's ordering (Sec. 3.3, Tables 3-4) through the whole path --------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_sloan_ordering_solve_matches_oracle(prec):
    import efie_problem as ep
    P = ep.build("plate1160")
    nl = len(P.leaf_ptr) - 1
    order = ordering.sloan(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    F = schur.setup(P, order, fill_tol=0.0)
    S = krylov.System(P, F)
    h = hm.hmat_create(P, ordering=2, fill_tol=0.0, precision=prec)
    hm.precond_setup(h)
    assert np.array_equal(hm.hm_get_order(h), order)
    ptr, idx = hm.hm_get_fill(h)
    for k in range(F.nb):
        assert list(idx[ptr[k]:ptr[k + 1]]) == F.S[k]
    b = P.plane_wave([0.6, 0.0, -0.8], [0.8, 0.0, 0.6])
    if prec == 0:
        for k in range(0, F.nb, 3):
            nk = int(F.size[k])
            assert rel(hm.hm_get_block(h, 0, k, (nk, nk)), F.D[k]) < 1e-10, k
        x, it, rr, code = hm.solve(h, b, tol=1e-6, restart=50)
        xo, ito, rro, ok = krylov.solve(S, b, tol=1e-6, restart=50)
        assert code == 0 and ok and abs(int(it[0]) - ito) <= 1
        assert rel(x, xo) <= 1e-8
    else:
        x, it, rr, code = hm.solve(h, b, tol=1e-5, restart=50)
        xt = krylov.solve(S, b, tol=1e-10, restart=50)[0]
        assert code == 0
        assert np.linalg.norm(b - S.Z_orig(x)) / np.linalg.norm(b) <= 1.01e-5
        assert rel(x, xt) <= 1e-4


# ---- the complex-FP32 far field: CUDA cores (kind 1) and tensor cores (kind 2) -------------------
def test_far_schedules_match_oracle(cfg1, cfg1_mixed):
    P, order, F, S, h64 = cfg1
    h = cfg1_mixed
    rng = np.random.default_rng(13)
    op = hm.hmsolve.OP32 + hm.hmsolve.OP_ZF
    for nrhs in (1, 5, 64):
        X = rng.standard_normal((S.n, nrhs)) + 1j * rng.standard_normal((S.n, nrhs))
        ref = np.stack([S.far_new(X[:, c]) for c in range(nrhs)], axis=1)
        res = {}
        for kind in (1, 2):
            hm.hmsolve.hm_set_far_schedule(h, kind)
            dy = torch.empty_like(_dev(X))
            hm.hm_apply(h, op, _dev(X), dy)
            res[kind] = _host(dy)
            for c in range(nrhs):          # FP32 factors and arithmetic against the FP64 oracle
                assert rel(res[kind][:, c], ref[:, c]) < 1e-5, (kind, nrhs, c)
        if nrhs > 1:                       # a column alone gives the same bits as in the batch
            for kind in (1, 2):
                hm.hmsolve.hm_set_far_schedule(h, kind)
                dy = torch.empty_like(_dev(X[:, :1]))
                hm.hm_apply(h, op, _dev(X[:, 3:4]), dy)
                assert np.array_equal(_host(dy)[:, 0], res[kind][:, 3]), kind
    hm.hmsolve.hm_set_far_schedule(h, 0)


# ---- block Jacobi (the block diagonal comparison preconditioner of Sec. 1) ----------------------
@pytest.mark.parametrize("which", ["small", "cfg1"])
def test_block_jacobi_matches_oracle(which, request):
    P, order, F, S, h = request.getfixturevalue(which)
    B = krylov.BlockJacobi(P, order)
    g = hm.hmat_create(P, ordering=1, preconditioner=1)
    hm.precond_setup(g)
    for k in range(0, F.nb, 3):
        nk = int(F.size[k])
        assert rel(hm.hm_get_block(g, 0, k, (nk, nk)), B.M[k]) < 1e-14, k
        assert rel(hm.hm_get_block(g, 1, k, (nk, nk)), np.linalg.inv(B.M[k])) < 1e-9, k
    rng = np.random.default_rng(23)
    X = rng.standard_normal((S.n, 3)) + 1j * rng.standard_normal((S.n, 3))
    for op, f in ((hm.hmsolve.OP_A, B.apply_A), (hm.hmsolve.OP_DINV, B.M_solve),
                  (hm.hmsolve.OP_LINV, lambda x: x), (hm.hmsolve.OP_LTINV, lambda x: x)):
        dy = torch.empty_like(_dev(X))
        hm.hm_apply(g, op, _dev(X), dy)
        Y = _host(dy)
        for c in range(3):
            assert rel(Y[:, c], f(X[:, c])) < 1e-10, (op, c)
    # block Jacobi converges slowly on the EFIE (GMRES(30): 90 steps to 1e-4 on the 480-unknown
    # sphere, 1579 on the 1920-unknown one); GMRES(100) keeps the test short
    b = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    x, it, rr, code = hm.solve(g, b, tol=1e-4, restart=100, maxit=3000)
    xo, ito, rro, ok = krylov.solve(B, b, tol=1e-4, restart=100, maxit=3000)
    assert code == 0 and ok and abs(int(it[0]) - ito) <= 1
    assert rel(x, xo) <= 1e-8
    with pytest.raises(hm.HMError):
        hm.precond_setup(hm.hmat_create(P, ordering=1, preconditioner=1, precision=1))


# ---- null field (the one-sided comparison of Sec. 3 / Sec. 5.2: elimination without fill) --------
@pytest.mark.parametrize("which", ["small", "cfg1"])
def test_null_field_matches_oracle(which, request):
    P, order, F, S, h = request.getfixturevalue(which)
    N = krylov.NullField(P, order)
    g = hm.hmat_create(P, ordering=1, preconditioner=2, fill_tol=1e-2)
    hm.precond_setup(g)
    ptr, idx = hm.hm_get_fill(g)
    assert ptr[-1] < len(hm.hm_get_fill(h)[1])            # the Schur factor of this order fills
    for k in range(N.F.nb):
        assert list(idx[ptr[k]:ptr[k + 1]]) == N.F.S[k]
    assert np.all(hm.hmsolve.hm_get_fill_ranks(g) == -1)   # nothing to compress without fill
    st = hm.hmat_stats(g)
    assert st["coef_entries"] == st["coef_entries_dense"]
    for k in range(N.F.nb):
        nk = int(N.F.size[k])
        assert rel(hm.hm_get_block(g, 0, k, (nk, nk)), N.F.D[k]) < 1e-10, k
        assert rel(hm.hm_get_block(g, 1, k, (nk, nk)), np.linalg.inv(N.F.D[k])) < 1e-9, k
        if N.F.S[k]:
            M = int(sum(N.F.size[j] for j in N.F.S[k]))
            Wo = np.concatenate([N.F.W[(k, j)] for j in N.F.S[k]], axis=1)
            assert rel(hm.hm_get_block(g, 2, k, (nk, M)), Wo) < 1e-10, k
    rng = np.random.default_rng(24)
    X = rng.standard_normal((S.n, 3)) + 1j * rng.standard_normal((S.n, 3))
    for op, f in ((hm.hmsolve.OP_A, N.apply_A), (hm.hmsolve.OP_DINV, N.D_solve),
                  (hm.hmsolve.OP_LINV, N.L_inv), (hm.hmsolve.OP_LTINV, N.LT_inv)):
        dy = torch.empty_like(_dev(X))
        hm.hm_apply(g, op, _dev(X), dy)
        Y = _host(dy)
        for c in range(3):
            assert rel(Y[:, c], f(X[:, c])) < 1e-10, (op, c)
    b = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    x, it, rr, code = hm.solve(g, b, tol=1e-6, restart=30, maxit=3000)
    xo, ito, rro, ok = krylov.solve(N, b, tol=1e-6, restart=30, maxit=3000)
    assert code == 0 and ok and abs(int(it[0]) - ito) <= 1
    assert rel(x, xo) <= 1e-8
    # a column in a batch gives the bits of its solo solve
    B = np.stack([b, P.plane_wave([1.0, 0.0, 0.0], [0.0, 0.0, 1.0])], axis=1)
    xb, itb, rrb, codeb = hm.solve(g, B, tol=1e-6, restart=30, maxit=3000)
    assert np.array_equal(xb[:, 0], x) and int(itb[0]) == int(it[0])
    with pytest.raises(hm.HMError):
        hm.hmat_create(P, ordering=1, preconditioner=2, precision=1)


# ---- Sec. 3.4, compression during the setup (the abstract's reading) -----------------------------
def test_compression_in_setup_matches_oracle(sphere1920):
    P = sphere1920
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    F = schur.setup(P, order, fill_tol=1e-2, compress_in_setup=True)
    S = krylov.System(P, F)
    h = hm.hmat_create(P, ordering=1, fill_tol=1e-2, compress_in_setup=1)
    hm.precond_setup(h)
    ranks = hm.hmsolve.hm_get_fill_ranks(h)
    assert np.array_equal(ranks, [F.rank.get((k, j), -1) for k in range(F.nb) for j in F.S[k]])
    assert np.sum(ranks >= 0) > 0
    for k in range(F.nb):
        nk = int(F.size[k])
        assert rel(hm.hm_get_block(h, 0, k, (nk, nk)), F.D[k]) < 1e-8, k
        if F.S[k]:
            M = int(sum(F.size[j] for j in F.S[k]))
            Wo = np.concatenate([F.Wc[(k, j)] for j in F.S[k]], axis=1)
            assert rel(hm.hm_get_block(h, 2, k, (nk, M)), Wo) < 1e-8, k
    # the readings differ: the later pivot blocks see the truncated updates
    Fa = schur.setup(P, order, fill_tol=1e-2)
    assert max(rel(F.D[k], Fa.D[k]) for k in range(F.nb)) > 1e-6
    b = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    x, it, rr, code = hm.solve(h, b, tol=1e-6, restart=30)
    xo, ito, rro, ok = krylov.solve(S, b, tol=1e-6, restart=30)
    assert code == 0 and ok and abs(int(it[0]) - ito) <= 1
    assert rel(x, xo) <= 1e-8
