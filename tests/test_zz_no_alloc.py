"""hm_far_apply_noalloc: the far-field product for callers that must not allocate device
memory during the call (cudaFree synchronises the whole device; memory held in another
allocator's pool can make cudaMalloc fail).  Its output must match the regular far-field
product (hm_apply op 3) on two calls in a row, which share the library's static scratch."""
import numpy as np
import pytest
import torch

import paper_2111_13483_gb300 as hm

pytestmark = pytest.mark.gpu


def test_noalloc_far_product_matches_regular_path(sphere1920):
    h = hm.hmat_create(sphere1920, ordering=1)
    rng = np.random.default_rng(21)
    for call, nrhs in enumerate((3, 2)):          # two calls in a row, different shapes
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


def test_noalloc_rejects_calls_beyond_the_static_scratch(sphere1920):
    h = hm.hmat_create(sphere1920, ordering=1)
    nrhs = 600                                    # 1920 * 600 entries alone exceed 2^20
    dx = torch.zeros((nrhs, h.n), dtype=torch.complex128, device="cuda")
    dy = torch.zeros_like(dx)
    assert hm.hmsolve.hm_far_apply_noalloc(h, dx, dy) == hm.hmsolve.HM_EINVAL
    assert "static scratch" in hm.hm_last_error(h)
