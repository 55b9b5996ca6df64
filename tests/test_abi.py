"""C-ABI checks that need no GPU: the library builds and loads, exports every function
include/hmsolve.h declares, its host planner reproduces the oracle's ordering and fill,
and malformed descriptions are rejected with HM_EINVAL before any device work."""
import ctypes
import os
import re
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import ordering, schur

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hm():
    import paper_2111_13483_gb300 as pkg
    pkg.hmsolve.load()
    return pkg.hmsolve


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hmsolve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char \*)\s*\**\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(hm):
    lib = ctypes.CDLL(hm.lib_path())
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(hm.EXPORTS)


def test_default_opts(hm):
    o = hm.hm_opts()
    assert hm.load().hm_default_opts(ctypes.byref(o)) == 0
    assert o.ordering == 1 and o.fill_tol == 0.0 and o.precision == 0 and o.stream is None


def test_planner_order_and_fill_match_oracle(hm, sphere1920, sphere480):
    for P in (sphere480, sphere1920):
        nl = len(P.leaf_ptr) - 1
        pairs = list(zip(P.near_t.tolist(), P.near_s.tolist()))
        o = hm.hm_plan_order(nl, P.near_t, P.near_s)
        assert np.array_equal(o, ordering.rcm(nl, pairs))
        pos = np.empty(nl, dtype=np.int64)
        pos[o] = np.arange(nl)
        pi, pj = pos[P.near_t], pos[P.near_s]
        assert hm.hm_plan_fill(nl, pi, pj) == schur.symbolic_fill(nl, list(zip(pi.tolist(), pj.tolist())))


def test_planner_random_graphs_match_oracle(hm):
    rng = np.random.default_rng(11)
    for n in (1, 2, 7, 40, 130):
        m = rng.integers(0, 3 * n + 1)
        t = rng.integers(0, n, m)
        s = rng.integers(0, n, m)
        pairs = list(zip(t.tolist(), s.tolist()))
        o = hm.hm_plan_order(n, t, s)
        assert np.array_equal(o, ordering.rcm(n, pairs))
        assert hm.hm_plan_fill(n, t, s) == schur.symbolic_fill(n, pairs)


def test_planner_no_fill_lists_match_oracle(hm, sphere1920):
    """The null-field lists (closure 0: the later near-field neighbours only) equal the
    oracle's, on random graphs and on the 1920-unknown sphere in RCM order, and are contained
    in the symbolic fill; other closure values are rejected."""
    rng = np.random.default_rng(12)
    for n in (1, 2, 7, 40, 130):
        m = rng.integers(0, 3 * n + 1)
        t = rng.integers(0, n, m)
        s = rng.integers(0, n, m)
        pairs = list(zip(t.tolist(), s.tolist()))
        got = hm.hm_plan_fill(n, t, s, closure=0)
        assert got == schur.near_lists(n, pairs)
        full = hm.hm_plan_fill(n, t, s)
        assert all(set(a) <= set(b) for a, b in zip(got, full))
    P = sphere1920
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    pos = np.empty(nl, dtype=np.int64)
    pos[order] = np.arange(nl)
    bi, bj = pos[P.near_t], pos[P.near_s]
    pairs = list(zip(bi.tolist(), bj.tolist()))
    got = hm.hm_plan_fill(nl, bi, bj, closure=0)
    assert got == schur.near_lists(nl, pairs)
    assert sum(map(len, got)) < sum(map(len, hm.hm_plan_fill(nl, bi, bj)))
    with pytest.raises(hm.HMError):
        hm.hm_plan_fill(3, [0, 1], [1, 2], closure=2)


def test_planner_sloan_matches_oracle(hm, sphere1920, sphere480):
    import efie_problem as ep
    for P in (sphere480, sphere1920, ep.build("plate1160")):
        nl = len(P.leaf_ptr) - 1
        pairs = list(zip(P.near_t.tolist(), P.near_s.tolist()))
        assert np.array_equal(hm.hm_plan_order_method(2, nl, P.near_t, P.near_s), ordering.sloan(nl, pairs))
        assert np.array_equal(hm.hm_plan_order_method(1, nl, P.near_t, P.near_s), ordering.rcm(nl, pairs))
        assert np.array_equal(hm.hm_plan_order_method(0, nl, P.near_t, P.near_s), np.arange(nl))
    rng = np.random.default_rng(12)
    for n in (1, 2, 7, 40, 130):
        m = rng.integers(0, 3 * n + 1)
        t = rng.integers(0, n, m)
        s = rng.integers(0, n, m)
        assert np.array_equal(hm.hm_plan_order_method(2, n, t, s), ordering.sloan(n, list(zip(t.tolist(), s.tolist()))))
    with pytest.raises(hm.HMError):
        hm.hm_plan_order_method(3, 4, [0], [1])


def test_planner_rejects_bad_input(hm):
    with pytest.raises(hm.HMError):
        hm.hm_plan_order(3, [0, 5], [1, 1])
    with pytest.raises(hm.HMError):
        hm.hm_plan_fill(3, [0, -1], [1, 1])


def _tiny_problem():
    # 2 leaves of 2 unknowns, all near, symmetric blocks
    z = np.arange(1, 5, dtype=np.complex128)
    return SimpleNamespace(perm=np.array([0, 1, 2, 3]), leaf_ptr=np.array([0, 2, 4]), near_t=np.array([0, 0, 1]),
                           near_s=np.array([0, 1, 1]), near_off=np.array([0, 4, 8]),
                           near_data=np.concatenate([z, z, z]), far_r0=np.zeros(0), far_r1=np.zeros(0),
                           far_c0=np.zeros(0), far_c1=np.zeros(0), far_rank=np.zeros(0), far_uoff=np.zeros(0),
                           far_voff=np.zeros(0), far_U=np.zeros(0, np.complex128), far_V=np.zeros(0, np.complex128))


@pytest.mark.parametrize("breakage", ["perm", "leaf_ptr", "missing_diag", "t_gt_s", "dup", "offset", "coverage",
                                      "leaf_too_big"])
def test_create_rejects_malformed_descriptions(hm, breakage):
    p = _tiny_problem()
    if breakage == "perm":
        p.perm = np.array([0, 1, 1, 3])
    elif breakage == "leaf_ptr":
        p.leaf_ptr = np.array([0, 2, 5])
    elif breakage == "missing_diag":
        p.near_t, p.near_s, p.near_off = np.array([0, 0]), np.array([0, 1]), np.array([0, 4])
    elif breakage == "t_gt_s":
        p.near_t, p.near_s = np.array([0, 1, 1]), np.array([0, 0, 1])
    elif breakage == "dup":
        p.near_t, p.near_s = np.array([0, 0, 0, 1]), np.array([0, 1, 1, 1])
        p.near_off = np.array([0, 4, 4, 8])
    elif breakage == "offset":
        p.near_off = np.array([0, 4, 10])
    elif breakage == "coverage":
        p.near_t, p.near_s, p.near_off = np.array([0, 1]), np.array([0, 1]), np.array([0, 4])
    elif breakage == "leaf_too_big":
        n = 65
        p.perm = np.arange(n)
        p.leaf_ptr = np.array([0, n])
        p.near_t, p.near_s, p.near_off = np.array([0]), np.array([0]), np.array([0])
        p.near_data = np.zeros(n * n, np.complex128)
    with pytest.raises(hm.HMError) as ei:
        hm.hmat_create(p)
    assert ei.value.code == hm.HM_EINVAL


@pytest.mark.parametrize("opts", [dict(preconditioner=3), dict(preconditioner=-1), dict(preconditioner=1, precision=1),
                                  dict(preconditioner=2, precision=1), dict(ordering=3), dict(precision=2),
                                  dict(fill_tol=-1.0), dict(compress_in_setup=2)])
def test_create_rejects_bad_options(hm, opts):
    """Option values outside their ranges, and the comparison preconditioners (block Jacobi,
    null field) with the mixed precision, are rejected before any device work."""
    with pytest.raises(hm.HMError) as ei:
        hm.hmat_create(_tiny_problem(), **opts)
    assert ei.value.code == hm.HM_EINVAL


@pytest.mark.parametrize("breakage", ["row_index", "col_index", "empty_block", "mirror", "triangle", "free_vertex",
                                      "wavenumber", "eps"])
def test_efie_calls_reject_bad_arguments_before_any_device_work(hm, breakage):
    """hm_efie_fill / hm_efie_far validate every index and size on the host (HM_EINVAL) before
    touching a device, so these run without a GPU."""
    import efie_problem as ep
    import efie_problem.builder as B
    H = hm
    P = ep.build("plate_tiny")
    V, T, tri, free = P.rwg.V, P.rwg.T.copy(), P.rwg.tri.copy(), P.rwg.free.copy()
    k, rows, cols, mirror, eps = B.K0, [np.array([0, 1])], [np.array([2])], 0, 1e-3
    if breakage == "row_index":
        rows = [np.array([0, P.n])]
    elif breakage == "col_index":
        cols = [np.array([-1])]
    elif breakage == "empty_block":
        rows = [np.zeros(0, np.int32)]
    elif breakage == "mirror":
        mirror = 2
    elif breakage == "triangle":
        tri[0, 1] = len(T)
    elif breakage == "free_vertex":
        free[3, 0] = len(V)
    elif breakage == "wavenumber":
        k = 0.0
    elif breakage == "eps":
        eps = 1.5
    mesh = H.Mesh(V, T, tri, free, k, B.ETA0)
    with pytest.raises(hm.HMError) as ei:
        if breakage == "eps":
            H.hm_efie_far(mesh, rows, cols, eps)
        else:
            H.hm_efie_fill(mesh, rows, cols, mirror=mirror)
    assert ei.value.code == H.HM_EINVAL
    if breakage not in ("mirror", "eps"):
        with pytest.raises(hm.HMError) as ei:
            H.hm_efie_far(mesh, rows, cols, 1e-3)
        assert ei.value.code == H.HM_EINVAL


def test_efie_calls_accept_no_blocks(hm):
    import efie_problem as ep
    import efie_problem.builder as B
    H = hm
    P = ep.build("plate_tiny")
    mesh = H.Mesh(P.rwg.V, P.rwg.T, P.rwg.tri, P.rwg.free, B.K0, B.ETA0)
    out, off = H.hm_efie_fill(mesh, [], [])
    assert len(out) == 0 and list(off) == [0]
    rank, uoff, voff, U, Vf = H.hm_efie_far(mesh, [], [], 1e-3)
    assert len(rank) == 0 and len(U) == 0 and len(Vf) == 0
