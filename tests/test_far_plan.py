"""The far-field plan of the library (hm_plan_far: phase-1 rank-vector tasks, phase-2
contraction segments, per-leaf parts) replayed on the CPU with numpy, exactly as the kernels
address memory, against Z_F u assembled densely from the problem's far blocks (Eqs. 8-11:
U V^T for low-rank blocks, the stored block for dense ones, the (c, r) block the transpose of
the (r, c) one).  Host logic only: no GPU."""
import numpy as np
import pytest

import paper_2111_13483_gb300 as hm


def dense_far(P):
    n = P.n
    Z = np.zeros((n, n), dtype=np.complex128)
    for b in range(len(P.far_rank)):
        r0, r1, c0, c1, r = (int(P.far_r0[b]), int(P.far_r1[b]), int(P.far_c0[b]), int(P.far_c1[b]),
                             int(P.far_rank[b]))
        m, c = r1 - r0, c1 - c0
        uo, vo = int(P.far_uoff[b]), int(P.far_voff[b])
        if r < 0:
            D = P.far_U[uo:uo + m * c].reshape(c, m).T
        else:
            U = P.far_U[uo:uo + m * r].reshape(r, m).T
            V = P.far_V[vo:vo + c * r].reshape(r, c).T
            D = U @ V.T
        Z[r0:r1, c0:c1] = D
        Z[c0:c1, r0:r1] = D.T
    return Z


def replay(P, plan, u):
    """Phase 1 then phase 2 of the far-field product, following the plan's tables."""
    items, tasks = plan["items"], plan["tasks"]
    tlen = int((items[:, 3] + items[:, 2]).max()) if len(items) else 0
    t = np.zeros(tlen, dtype=np.complex128)
    s = np.zeros(tlen, dtype=np.complex128)
    written = np.zeros((2, tlen), dtype=np.int64)
    for lo, hi, i0, i1 in tasks:
        for off, ld, rank, row, isv in items[i0:i1]:
            F = P.far_V if isv else P.far_U
            for l in range(rank):
                vec = F[off + l * ld: off + l * ld + (hi - lo)]
                (t if isv else s)[row + l] = vec @ u[lo:hi]
                written[isv, row + l] += 1
    y = np.zeros(P.n, dtype=np.complex128)
    src_vec = [t, s, u]
    for l in range(len(P.leaf_ptr) - 1):
        a, ni = int(P.leaf_ptr[l]), int(P.leaf_ptr[l + 1] - P.leaf_ptr[l])
        for foff, yrow, fi, fk, ln, src in plan["segs"][plan["seg_ptr"][l]:plan["seg_ptr"][l + 1]]:
            F = P.far_V if src & 1 else P.far_U
            idx = foff + np.arange(ni)[:, None] * fi + np.arange(ln)[None, :] * fk
            y[a:a + ni] += F[idx] @ src_vec[src >> 1][yrow:yrow + ln]
    return y, written


@pytest.fixture(scope="module")
def far_case(sphere1920):
    P = sphere1920
    assert (P.far_rank >= 0).any() and (P.far_rank < 0).any()   # both kinds of far block
    return P, hm.hmsolve.hm_plan_far(P)


def test_replayed_plan_is_the_far_field_product(far_case):
    P, plan = far_case
    rng = np.random.default_rng(11)
    u = rng.standard_normal(P.n) + 1j * rng.standard_normal(P.n)
    y, written = replay(P, plan, u)
    ref = dense_far(P) @ u
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
    # every rank vector entry is computed exactly once (t from V over the column range,
    # s from U over the row range)
    need = int(np.sum(np.maximum(P.far_rank, 0)))
    assert written.shape[1] == need and np.all(written == 1)


def test_segments_and_parts(far_case):
    P, plan = far_case
    segs, seg_ptr, part_ptr = plan["segs"], plan["seg_ptr"], plan["part_ptr"]
    nl = len(P.leaf_ptr) - 1
    assert seg_ptr[0] == 0 and seg_ptr[-1] == len(segs) and np.all(np.diff(seg_ptr) >= 0)
    assert np.all((segs[:, 4] >= 1) & (segs[:, 4] <= 32))                 # contraction pieces of <= 32
    parts = (len(part_ptr) - 1) // nl
    assert parts * nl + 1 == len(part_ptr) and parts >= 1
    kcum = np.concatenate([[0], np.cumsum(segs[:, 4])])
    for l in range(nl):
        pp = list(part_ptr[l * parts:(l + 1) * parts]) + [part_ptr[(l + 1) * parts]]
        assert pp[0] == seg_ptr[l] and pp[-1] == seg_ptr[l + 1] and all(np.diff(pp) >= 0)
        K = kcum[seg_ptr[l + 1]] - kcum[seg_ptr[l]]
        for p in range(parts):   # parts of about equal contraction length (segments are <= 32)
            assert kcum[pp[p + 1]] - kcum[pp[p]] <= K / parts + 32


def test_bad_descriptions_rejected(far_case):
    P, _ = far_case

    class Q:
        pass

    q = Q()
    for f in ("n", "leaf_ptr", "far_r0", "far_r1", "far_c0", "far_c1", "far_rank", "far_uoff", "far_voff"):
        setattr(q, f, getattr(P, f))
    q.far_r0 = np.array(P.far_r0).copy()
    q.far_r0[0] += 1                                   # not a leaf boundary
    with pytest.raises(hm.HMError):
        hm.hmsolve.hm_plan_far(q)
    q.far_r0 = P.far_r0
    q.far_rank = np.array(P.far_rank).copy()
    q.far_rank[0] = 10 ** 6                            # rank above min(m, c)
    with pytest.raises(hm.HMError):
        hm.hmsolve.hm_plan_far(q)
