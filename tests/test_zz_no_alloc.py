"""hm_far_apply_noalloc: the far-field product for callers that must not allocate device
memory during the call (cudaFree synchronises the whole device; memory held in another
allocator's pool can make cudaMalloc fail).  Its output must match the regular far-field
product (hm_apply op 3) on two calls in a row, which share the library's static scratch."""
import numpy as np
import pytest
import torch

import paper_2111_13483_gb300 as hm

pytestmark = pytest.mark.gpu

SCRATCH_ENTRIES = 1 << 20   # the static array's size in complex doubles (see the header)


def _two_calls(h, shapes, seed):
    rng = np.random.default_rng(seed)
    for call, nrhs in enumerate(shapes):          # calls in a row, different shapes
        X = rng.standard_normal((nrhs, h.n)) + 1j * rng.standard_normal((nrhs, h.n))
        dx = torch.from_numpy(X).cuda()
        y_ref = torch.empty_like(dx)
        y_na = torch.full_like(dx, complex(np.nan, np.nan))
        hm.hm_apply(h, hm.hmsolve.OP_ZF, dx, y_ref)
        code = hm.hmsolve.hm_far_apply_noalloc(h, dx, y_na)
        torch.cuda.synchronize()
        assert code == hm.hmsolve.HM_OK, hm.hm_last_error(h)
        a, b = y_na.cpu().numpy(), y_ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), call


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_noalloc_far_product_matches_regular_path(sphere1920, prec):
    """Both handle kinds keep the FP64 far factors the call reads (a precision 1 handle also
    holds FP32 copies for its inner operator)."""
    h = hm.hmat_create(sphere1920, ordering=1, precision=prec)
    _two_calls(h, (3, 2), 21 + prec)


def test_noalloc_full_size_sphere_one_rhs_per_call(sphere30720):
    """The 30,720-unknown sphere fits the static scratch at one right-hand side per call:
    n + 2 sum(rank) entries <= 2^20, and the product matches the regular path."""
    P = sphere30720
    need = P.n + 2 * int(np.sum(np.maximum(P.far_rank, 0)))
    assert need <= SCRATCH_ENTRIES < 2 * need
    h = hm.hmat_create(P, ordering=1)
    _two_calls(h, (1, 1), 23)
    dx = torch.zeros((2, h.n), dtype=torch.complex128, device="cuda")
    assert hm.hmsolve.hm_far_apply_noalloc(h, dx, torch.zeros_like(dx)) == hm.hmsolve.HM_EINVAL


def test_noalloc_rejects_calls_beyond_the_static_scratch(sphere1920):
    h = hm.hmat_create(sphere1920, ordering=1)
    nrhs = 600                                    # 1920 * 600 entries alone exceed 2^20
    dx = torch.zeros((nrhs, h.n), dtype=torch.complex128, device="cuda")
    dy = torch.zeros_like(dx)
    assert hm.hmsolve.hm_far_apply_noalloc(h, dx, dy) == hm.hmsolve.HM_EINVAL
    assert "static scratch" in hm.hm_last_error(h)
