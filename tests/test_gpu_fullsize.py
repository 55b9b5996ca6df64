"""GPU parity at the sizes and launch shapes of the benchmark.

7,680-unknown sphere (272 blocks): everything against the oracle.  The operators run at 64
right-hand-side columns with the tuned sweep schedule, i.e. 272 block rows x column groups
of CTAs against the resident slots of the GPU, so the ticket-ordered waits across CTAs that
are not yet resident are exercised; 16 sampled columns are compared with the oracle element
by element, and every column with its own one-column launch (bitwise, batch invariance).

30,720-unknown sphere (1,112 blocks, the benchmark problem): what the oracle computes in
seconds at this size -- order and fill, the first elimination steps, sampled far-field
columns -- plus properties that hold at any size:
* Eq. 21: L^{-1} Z_N L^{-T} = D, checked as L^{-1} (Z_N (L^{-T} X)) = D X for 64 columns,
  with Z_N X taken by the oracle from the near blocks as ingested; this reaches every block
  row of both sweeps, the ~230-dependency rows included, at the benchmark's launch width;
* the mixed-precision solve's true residual ||V - Z I|| / ||V||, with Z applied by the oracle.

Tolerances: FP64 1e-10 (operators, factor blocks; 1e-9 for explicit inverses), FP64
solutions 1e-8 with iteration counts +-1; the identity 1e-11 (it holds to 2e-15 with the
oracle's own factors on these meshes); complex-FP32 operators 1e-4 against FP64 (FP32
factors and arithmetic over contractions of up to ~7,000 terms); mixed solutions 1e-4
against the oracle's tol-1e-10 solve, mixed residual at the requested 1e-5.
"""
import numpy as np
import pytest
import torch

import paper_2111_13483_gb300 as hm
from oracle import krylov, ordering, schur
from refs import truncated_at

pytestmark = pytest.mark.gpu
H = hm.hmsolve


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def elem_ok(y, ref, tol):
    """Element by element: |y_i - ref_i| <= tol * max_i |ref_i|."""
    return np.max(np.abs(y - ref)) <= tol * np.max(np.abs(ref))


def _dev(X):            # X: n x c (solve order) -> device (c, n)
    return torch.from_numpy(np.ascontiguousarray(X.T)).cuda()


def _apply(h, op, X):
    dx = _dev(X)
    dy = torch.empty_like(dx)
    hm.hm_apply(h, op, dx, dy)
    return dy.cpu().numpy().T


def _rand(n, c, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, c)) + 1j * rng.standard_normal((n, c))


# ---- 7,680 unknowns: full oracle comparison --------------------------------------------
@pytest.fixture(scope="module")
def s7680(sphere7680):
    P = sphere7680
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    F = schur.setup(P, order, fill_tol=0.0)
    S = krylov.System(P, F)
    h64 = hm.hmat_create(P, ordering=1, precision=0)
    hm.precond_setup(h64)
    h32 = hm.hmat_create(P, ordering=1, precision=1)
    hm.precond_setup(h32)
    return P, order, F, S, h64, h32


def test_7680_order_fill_and_blocks(s7680):
    P, order, F, S, h64, h32 = s7680
    assert np.array_equal(hm.hm_get_order(h64), order)
    assert np.array_equal(hm.hm_get_order(h32), order)
    ptr, idx = hm.hm_get_fill(h64)
    for k in range(F.nb):
        assert list(idx[ptr[k]:ptr[k + 1]]) == F.S[k]
    assert np.array_equal(hm.hm_get_index_map(h64), S.new2orig)
    assert max(len(s) for s in F.S) > 40          # heavy rows are present at this size
    for k in list(range(0, F.nb, 7)) + [F.nb - 1]:
        nk = int(F.size[k])
        assert rel(hm.hm_get_block(h64, 0, k, (nk, nk)), F.D[k]) < 1e-10, k
        assert rel(hm.hm_get_block(h64, 1, k, (nk, nk)), np.linalg.inv(F.D[k])) < 1e-9, k
        if F.S[k]:
            M = int(sum(F.size[j] for j in F.S[k]))
            Wo = np.concatenate([F.W[(k, j)] for j in F.S[k]], axis=1)
            assert rel(hm.hm_get_block(h64, 2, k, (nk, M)), Wo) < 1e-10, k
            assert rel(hm.hm_get_block(h32, 2, k, (nk, M)), Wo) < 1e-4, k


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_7680_operators_64_columns(s7680, prec):
    P, order, F, S, h64, h32 = s7680
    h = h64 if prec == 0 else h32
    off = 0 if prec == 0 else H.OP32
    tol = 1e-10 if prec == 0 else 1e-4
    X = _rand(S.n, 64, 31 + prec)
    refs = {H.OP_LINV: S.L_inv, H.OP_LTINV: S.LT_inv, H.OP_ZF: S.far_new, H.OP_A: S.apply_A}
    sample = list(range(0, 64, 4))
    for op, f in refs.items():
        Y = _apply(h, off + op, X)
        for c in sample:
            ref = f(X[:, c])
            assert rel(Y[:, c], ref) < tol, (op, c)
            assert elem_ok(Y[:, c], ref, 10 * tol), (op, c)
        for c in range(0, 64, 9):   # batch invariance: each column equals its one-column launch
            assert np.array_equal(_apply(h, off + op, X[:, c:c + 1])[:, 0], Y[:, c]), (op, c)


@pytest.fixture(scope="module")
def s7680c(sphere7680):
    """The same sphere with the fill-in blocks compressed at fill_tol 1e-2 (Sec. 3.4), stored
    and applied as factors."""
    P = sphere7680
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    F = schur.setup(P, order, fill_tol=1e-2)
    S = krylov.System(P, F)
    h64 = hm.hmat_create(P, ordering=1, fill_tol=1e-2, precision=0)
    hm.precond_setup(h64)
    h32 = hm.hmat_create(P, ordering=1, fill_tol=1e-2, precision=1)
    hm.precond_setup(h32)
    return P, F, S, h64, h32


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_7680_compressed_operators_64_columns(s7680c, prec):
    P, F, S, h64, h32 = s7680c
    h = h64 if prec == 0 else h32
    off = 0 if prec == 0 else H.OP32
    tol = 1e-10 if prec == 0 else 1e-4
    if prec == 0:
        ranks = hm.hmsolve.hm_get_fill_ranks(h)
        ptr, idx = hm.hm_get_fill(h)
        expect = [F.rank.get((k, j), -1) for k in range(F.nb) for j in F.S[k]]
        assert np.array_equal(ranks, expect)
        assert hm.hmat_stats(h)["coef_entries"] == schur.nnz_coefficients(F) - int(np.sum(F.size))
    X = _rand(S.n, 64, 51 + prec)
    refs = [(H.OP_LINV, S.L_inv), (H.OP_LTINV, S.LT_inv), (H.OP_A, S.apply_A)]
    if prec == 1:   # the FP32 setup's ranks, truncated in FP64 (see truncated_at)
        Wm = truncated_at(F, h)
        refs = [(H.OP_LINV, lambda x: S.join(schur.sweep_forward(F, S.split(x), W=Wm))),
                (H.OP_LTINV, lambda x: S.join(schur.sweep_backward(F, S.split(x), W=Wm)))]
    for op, f in refs:
        Y = _apply(h, off + op, X)
        for c in range(0, 64, 8):
            assert rel(Y[:, c], f(X[:, c])) < tol, (op, c)
        for c in (5, 40):
            assert np.array_equal(_apply(h, off + op, X[:, c:c + 1])[:, 0], Y[:, c]), (op, c)


def test_7680_fp64_solve_matches_oracle(s7680):
    P, order, F, S, h64, h32 = s7680
    b = P.plane_wave([-1.0, 0.0, 0.0], [0.0, 0.0, -1.0])
    x, it, rr, code = hm.solve(h64, b, tol=1e-4, restart=30)
    xo, ito, rro, ok = krylov.solve(S, b, tol=1e-4, restart=30)
    assert code == 0 and ok and abs(int(it[0]) - ito) <= 1
    assert rel(x, xo) <= 1e-8


def test_7680_mixed_solve_within_1e4_of_tight_oracle(s7680):
    P, order, F, S, h64, h32 = s7680
    B = np.stack([P.plane_wave([-np.cos(p), -np.sin(p), 0.0], [0.0, 0.0, -1.0]) for p in (0.0, 2.0)], axis=1)
    I, its, rr, code = hm.solve(h32, B, tol=1e-5, restart=30)
    assert code == 0
    for c in range(B.shape[1]):
        xt, itt, rrt, ok = krylov.solve(S, B[:, c], tol=1e-10, restart=30)
        assert ok
        assert np.linalg.norm(B[:, c] - S.Z_orig(I[:, c])) / np.linalg.norm(B[:, c]) <= 1.01e-5
        assert rel(I[:, c], xt) <= 1e-4, c


# ---- 30,720 unknowns: the benchmark problem --------------------------------------------
NSTEPS = 48     # elimination steps the oracle runs (seconds) for the sampled factor checks


@pytest.fixture(scope="module")
def s30720(sphere30720):
    P = sphere30720
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    F = schur.setup(P, order, fill_tol=0.0, max_steps=NSTEPS)
    S = krylov.System(P, F)      # index maps only (order and sizes)
    h64 = hm.hmat_create(P, ordering=1, precision=0)
    hm.precond_setup(h64)
    h32 = hm.hmat_create(P, ordering=1, precision=1)
    hm.precond_setup(h32)
    return P, order, F, S, h64, h32


def test_30720_order_fill_and_first_steps(s30720):
    P, order, F, S, h64, h32 = s30720
    assert np.array_equal(hm.hm_get_order(h64), order)
    ptr, idx = hm.hm_get_fill(h64)
    for k in range(F.nb):                          # the oracle's symbolic fill is complete
        assert list(idx[ptr[k]:ptr[k + 1]]) == list(F.S[k]), k
    assert max(len(s) for s in F.S) > 150          # the heavy rows of the sweeps
    assert np.array_equal(hm.hm_get_index_map(h64), S.new2orig)
    for k in range(NSTEPS):
        nk = int(F.size[k])
        assert rel(hm.hm_get_block(h64, 0, k, (nk, nk)), F.D[k]) < 1e-10, k
        assert rel(hm.hm_get_block(h64, 1, k, (nk, nk)), np.linalg.inv(F.D[k])) < 1e-9, k
        if F.S[k]:
            M = int(sum(F.size[j] for j in F.S[k]))
            Wo = np.concatenate([F.W[(k, j)] for j in F.S[k]], axis=1)
            assert rel(hm.hm_get_block(h64, 2, k, (nk, M)), Wo) < 1e-10, k


def test_30720_far_field_64_columns(s30720):
    P, order, F, S, h64, h32 = s30720
    X = _rand(S.n, 64, 41)
    Y = _apply(h64, H.OP_ZF, X)
    for c in (0, 37, 63):
        ref = S.far_new(X[:, c])
        assert rel(Y[:, c], ref) < 1e-10, c
        assert elem_ok(Y[:, c], ref, 1e-9), c


def _near_solve_order(S, Y):
    """Z_N Y by the oracle from the ingested near blocks; Y in solve order (n x c)."""
    u = np.zeros(Y.shape, dtype=np.complex128)
    u[S.new2cl] = Y
    return S.near_cluster(u)[S.new2cl]


def _d_mul(h, S, X):
    """D X with the GPU's D_k (Eq. 21), block by block on the host."""
    out = np.empty_like(X)
    for k in range(S.F.nb):
        a, b = S.off[k], S.off[k + 1]
        out[a:b] = hm.hm_get_block(h, 0, k, (b - a, b - a)) @ X[a:b]
    return out


def test_30720_eq21_identity_64_columns(s30720):
    """L^{-1} Z_N L^{-T} X = D X (Eq. 21), both sweeps at the benchmark's 64-column width."""
    P, order, F, S, h64, h32 = s30720
    X = _rand(S.n, 64, 43)
    Y = _apply(h64, H.OP_LTINV, X)
    W = _apply(h64, H.OP_LINV, _near_solve_order(S, Y))
    DX = _d_mul(h64, S, X)
    for c in range(64):
        assert rel(W[:, c], DX[:, c]) < 1e-11, c


def test_30720_mixed_operators_and_solve(s30720):
    P, order, F, S, h64, h32 = s30720
    X = _rand(S.n, 64, 47)
    for op in (H.OP_LINV, H.OP_LTINV):
        Y64 = _apply(h64, op, X)
        Y32 = _apply(h32, H.OP32 + op, X)
        for c in range(64):
            assert rel(Y32[:, c], Y64[:, c]) < 1e-4, (op, c)
    b = P.plane_wave([0.0, -1.0, 0.0], [0.0, 0.0, -1.0])
    I, its, rr, code = hm.solve(h32, b, tol=1e-5, restart=30)
    assert code == 0 and rr[0] <= 1e-5
    assert np.linalg.norm(b - S.Z_orig(I)) / np.linalg.norm(b) <= 1.01e-5


@pytest.mark.parametrize("nrhs", [16, 64])
def test_7680_cluster_sweeps_bitwise_equal_compressed_mixed(s7680c, nrhs):
    """The cluster-chained sweeps (kinds 5, 6) at the benchmark's widths on a problem with more
    CTAs than resident slots and compressed fill-in blocks: bitwise the one-row-per-CTA result."""
    P, F, S, h64, h32 = s7680c
    X = _rand(S.n, nrhs, 71)
    try:
        for op in (H.OP32 + H.OP_LINV, H.OP32 + H.OP_LTINV):
            ref = None
            for sched in ((2, 1, 0), (1, 5, 0), (2, 5, 0), (4, 5, 0), (1, 6, 0), (2, 6, 0)):
                H.hm_set_sweep_schedule(h32, *sched)
                Y = _apply(h32, op, X)
                if ref is None:
                    ref = Y
                else:
                    assert np.array_equal(Y, ref), (sched, op)
    finally:
        H.hm_set_sweep_schedule(h32, 0, 0)
