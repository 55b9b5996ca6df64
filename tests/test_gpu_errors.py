"""Error paths of the C-ABI on the GPU, each produced on the host (no GPU fault, trap or hang):

* HM_ESINGULAR: a description whose first pivot block (Sec. 3.1, Eq. 14) is zero;
* HM_ENOMEM: an hbm_budget too small for hmat_create, and one that fits the upload but not
  the factors of precond_setup;
* HM_ETIMEOUT: the test hook leaves one block row of the triangular sweeps (Eqs. 23, 24) out,
  so the rows that depend on it wait on a result that is never published; with a 10 ms bound
  on every wait the operator returns HM_ETIMEOUT, and once the hook is cleared the same handle
  gives the same result as before.
"""
import copy

import numpy as np
import pytest
import torch

import paper_2111_13483_gb300 as hm

pytestmark = pytest.mark.gpu
H = hm.hmsolve


def _zero_first_pivot(P):
    """A copy of P whose near-field diagonal block of the leaf eliminated first is zero."""
    Q = copy.copy(P)
    nl = len(P.leaf_ptr) - 1
    order = hm.hm_plan_order(nl, P.near_t, P.near_s)
    l0 = int(order[0])
    b = int(np.nonzero((P.near_t == l0) & (P.near_s == l0))[0][0])
    m = int(P.leaf_ptr[l0 + 1] - P.leaf_ptr[l0])
    Q.near_data = P.near_data.copy()
    Q.near_data[P.near_off[b]:P.near_off[b] + m * m] = 0
    return Q


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("ctas", [1, 4])
def test_singular_pivot_block(sphere480, prec, ctas):
    Q = _zero_first_pivot(sphere480)
    h = hm.hmat_create(Q, ordering=1, precision=prec)
    hm.hmsolve.hm_set_pivot_schedule(h, ctas)
    with pytest.raises(hm.HMError) as ei:
        hm.precond_setup(h)
    assert ei.value.code == H.HM_ESINGULAR
    assert "D_0" in hm.hm_last_error(h)
    with pytest.raises(hm.HMError) as ei:      # no factors: the solve is refused
        hm.solve(h, Q.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0]))
    assert ei.value.code == H.HM_ESTATE
    hm.hmat_destroy(h)


def test_budget_too_small_for_create(sphere480):
    with pytest.raises(hm.HMError) as ei:
        hm.hmat_create(sphere480, ordering=1, hbm_budget=4096)
    assert ei.value.code == H.HM_ENOMEM


@pytest.mark.parametrize("prec", [0, 1])
def test_budget_too_small_for_setup(sphere480, prec):
    g = hm.hmat_create(sphere480, ordering=1, precision=prec)
    need = hm.hmat_stats(g)["device_bytes"]
    hm.hmat_destroy(g)
    h = hm.hmat_create(sphere480, ordering=1, precision=prec, hbm_budget=need + 4096)
    with pytest.raises(hm.HMError) as ei:
        hm.precond_setup(h)
    assert ei.value.code == H.HM_ENOMEM
    hm.hmat_destroy(h)


@pytest.fixture(scope="module", params=[0, 1], ids=["fp64", "mixed"])
def handle(request, sphere480):
    h = hm.hmat_create(sphere480, ordering=1, precision=request.param)
    hm.precond_setup(h)
    yield sphere480, h, request.param
    H.hm_test_hold(h, -1, 0)


def test_unpublished_block_times_out_and_handle_recovers(handle):
    P, h, prec = handle
    nb = h.n_leaves
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, P.n)) + 1j * rng.standard_normal((3, P.n))
    dx = torch.from_numpy(X).cuda()
    off = H.OP32 if prec == 1 else 0
    ref = {}
    for op in (H.OP_LINV, H.OP_LTINV, H.OP_A):
        dy = torch.empty_like(dx)
        hm.hm_apply(h, off + op, dx, dy)
        ref[op] = dy.cpu().numpy()
    # forward sweep: block row 0 comes first and (with RCM) later rows depend on it;
    # backward sweep: the last block row comes first
    for op, held in ((H.OP_LINV, 0), (H.OP_LTINV, nb - 1), (H.OP_A, 0)):
        H.hm_test_hold(h, held, 10_000_000)
        dy = torch.empty_like(dx)
        with pytest.raises(hm.HMError) as ei:
            hm.hm_apply(h, off + op, dx, dy)
        assert ei.value.code == H.HM_ETIMEOUT, op
        H.hm_test_hold(h, -1, 0)
        hm.hm_apply(h, off + op, dx, dy)
        assert np.array_equal(dy.cpu().numpy(), ref[op]), op


def test_cluster_sweeps_time_out_and_recover(handle):
    """The same with the cluster-chained sweeps (kind 5): a held row's in-cluster consumers
    give up on its ready word in shared memory, the others on its tagged words."""
    P, h, prec = handle
    nb = h.n_leaves
    rng = np.random.default_rng(6)
    dx = torch.from_numpy(rng.standard_normal((2, P.n)) + 1j * rng.standard_normal((2, P.n))).cuda()
    off = H.OP32 if prec == 1 else 0
    # rows whose result a later row of the same cluster (one group: sweep positions 0-7) reads:
    # forward, k in 1..6 with a row of S_k at most 7; backward, j >= nb - 7 in S_k of some
    # k >= nb - 8 below it
    sptr, sidx = H.hm_get_fill(h)
    S = [set(sidx[sptr[k]:sptr[k + 1]].tolist()) for k in range(nb)]
    fwd = next(k for k in range(1, 7) if any(j <= 7 for j in S[k]))
    bwd = next(j for j in range(nb - 2, nb - 8, -1) if any(j in S[k] for k in range(max(nb - 8, 0), j)))
    try:
        H.hm_set_sweep_schedule(h, 1, 5, 0)
        for op, held in ((H.OP_LINV, 0), (H.OP_LINV, fwd), (H.OP_LTINV, nb - 1), (H.OP_LTINV, bwd)):
            dy = torch.empty_like(dx)
            hm.hm_apply(h, off + op, dx, dy)
            ref = dy.cpu().numpy()
            H.hm_test_hold(h, held, 10_000_000)
            with pytest.raises(hm.HMError) as ei:
                hm.hm_apply(h, off + op, dx, dy)
            assert ei.value.code == H.HM_ETIMEOUT, (op, held)
            H.hm_test_hold(h, -1, 0)
            hm.hm_apply(h, off + op, dx, dy)
            assert np.array_equal(dy.cpu().numpy(), ref), (op, held)
    finally:
        H.hm_set_sweep_schedule(h, 0, 0)


def test_solve_times_out_then_succeeds(handle):
    P, h, prec = handle
    V = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    I0, it0, rr0, c0 = hm.solve(h, V, tol=1e-6)
    assert c0 == 0
    H.hm_test_hold(h, 0, 10_000_000)
    with pytest.raises(hm.HMError) as ei:
        hm.solve(h, V, tol=1e-6)
    assert ei.value.code == H.HM_ETIMEOUT
    H.hm_test_hold(h, -1, 0)
    I1, it1, rr1, c1 = hm.solve(h, V, tol=1e-6)
    assert c1 == 0 and it1[0] == it0[0] and np.array_equal(I1, I0)


def test_test_hold_rejects_bad_arguments(handle):
    P, h, prec = handle
    L = H.load()
    assert L.hm_test_hold(h.ptr, h.n_leaves, 0) == H.HM_EINVAL
    assert L.hm_test_hold(h.ptr, -2, 0) == H.HM_EINVAL
    assert L.hm_test_hold(h.ptr, 0, -1) == H.HM_EINVAL
    assert L.hm_test_hold(None, 0, 0) == H.HM_EINVAL
