"""Edge cases of the C-ABI path on the GPU: empty and zero right-hand sides, maxit = 0, state
errors, strided host buffers, more right-hand sides than engine slots, a tiny ragged problem."""
import numpy as np
import pytest
import torch

import paper_2111_13483_gb300 as hm
from oracle import krylov, ordering, schur

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.fixture(scope="module", params=[0, 1], ids=["fp64", "mixed"])
def small(request, sphere480):
    h = hm.hmat_create(sphere480, ordering=1, precision=request.param)
    hm.precond_setup(h)
    return sphere480, h, request.param


def test_zero_rhs_gives_zero_solution(small):
    P, h, prec = small
    V = np.zeros((P.n, 2), dtype=np.complex128)
    V[:, 1] = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    I, its, rr, code = hm.solve(h, V, tol=1e-6)
    assert code == 0
    assert np.all(I[:, 0] == 0) and its[0] == 0 and rr[0] == 0.0
    assert np.linalg.norm(I[:, 1]) > 0


def test_maxit_zero_reports_no_convergence(small):
    P, h, prec = small
    V = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    I, its, rr, code = hm.solve(h, V, tol=1e-6, maxit=0)
    assert code == hm.hmsolve.HM_ENOCONV
    assert its[0] == 0


def test_empty_batch_and_state_errors(small, sphere480):
    P, h, prec = small
    L = hm.hmsolve.load()
    iters = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1)
    assert L.solve(h.ptr, None, 0, P.n, 1e-4, 30, 100, None, P.n, iters.ctypes.data_as(hm.hmsolve._i32p),
                   rr.ctypes.data_as(hm.hmsolve._f64p)) == hm.hmsolve.HM_OK
    g = hm.hmat_create(sphere480, ordering=1, precision=prec)     # no precond_setup yet
    with pytest.raises(hm.HMError):
        hm.solve(g, P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0]))
    hm.hmat_destroy(g)
    if prec == 1:   # FP64 factor operators do not exist on a precision 1 handle
        x = torch.zeros(1, P.n, dtype=torch.complex128, device="cuda")
        with pytest.raises(hm.HMError):
            hm.hm_apply(h, hm.hmsolve.OP_LINV, x, torch.empty_like(x))


def test_strided_host_buffers(small):
    P, h, prec = small
    V = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    ref, it0, rr0, c0 = hm.solve(h, V, tol=1e-6)
    ld = P.n + 7
    Vs = np.zeros((2, ld), dtype=np.complex128)
    Vs[1, :P.n] = V
    Is = np.zeros((2, ld + 3), dtype=np.complex128)
    iters = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1)
    code = hm.hmsolve.load().solve(h.ptr, Vs[1].ctypes.data, 1, ld, 1e-6, 30, 5000, Is[1].ctypes.data, ld + 3,
                                   iters.ctypes.data_as(hm.hmsolve._i32p), rr.ctypes.data_as(hm.hmsolve._f64p))
    assert code == 0 and iters[0] == it0[0]
    assert np.array_equal(Is[1, :P.n], ref)
    assert np.all(Is[1, P.n:] == 0) and np.all(Is[0] == 0)


def test_more_columns_than_slots_equal_single_solves(small):
    """More right-hand sides than the engine's slots (64 mixed / 16 FP64): finished slots are
    refilled; every column still equals its single solve bitwise."""
    P, h, prec = small
    nrhs = 70 if prec == 1 else 20
    rng = np.random.default_rng(5)
    phis = rng.uniform(0, 2 * np.pi, nrhs)
    V = np.stack([P.plane_wave([-np.cos(p), -np.sin(p), 0.0], [0.0, 0.0, 1.0]) for p in phis], axis=1)
    I, its, rr, code = hm.solve(h, V, tol=1e-5)
    assert code == 0
    for c in (0, 17, nrhs - 1):
        x1, it1, rr1, c1 = hm.solve(h, V[:, c], tol=1e-5)
        assert it1[0] == its[c] and np.array_equal(x1, I[:, c]), c


def test_tiny_ragged_problem_matches_oracle():
    import efie_problem as ep
    P = ep.build("plate_tiny")          # leaves of 16, ragged sizes, few blocks
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    F = schur.setup(P, order, fill_tol=0.0)
    S = krylov.System(P, F)
    h = hm.hmat_create(P, ordering=1, fill_tol=0.0, precision=0)
    hm.precond_setup(h)
    assert np.array_equal(hm.hm_get_order(h), order)
    b = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    x, it, rr, code = hm.solve(h, b, tol=1e-8, restart=50)
    xo, ito, rro, ok = krylov.solve(S, b, tol=1e-8, restart=50)
    assert code == 0 and ok and abs(int(it[0]) - ito) <= 1
    assert rel(x, xo) <= 1e-8
