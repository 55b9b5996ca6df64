"""The tensor-core micro-kernel of the complex-FP32 sweeps (hm_tc_cgemm) against a plain
complex128 product.

Error bound per entry (3xTF32 with FP32 accumulation): with u = 2^-24, each FP32 input is
represented as hi + lo up to 2^-11 * 2^-11 of its value (TF32 keeps 10 fraction bits of the
remainder), the dropped lo*lo term is below 2^-22 of |a||b|, and the FP32 accumulation of k
terms adds at most a few k u; so |C - A B| <= (16 * 2^-22 + 8 k u) (|A| |B|) entrywise, with
|A| |B| the product of the entrywise moduli.  Plain TF32 products would miss this bound by
orders of magnitude (2^-11 per input); the test also checks the observed error sits at FP32
level.  Column independence: every column of C is bitwise the same for any number of columns.
"""
import numpy as np
import pytest
import torch

import paper_2111_13483_gb300 as hm

pytestmark = pytest.mark.gpu
H = hm.hmsolve


def _cg(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _run(A, B):
    """A (m x k), B (k x nc) complex64 host arrays -> C (m x nc) from the tensor cores."""
    m, k = A.shape
    nc = B.shape[1]
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    dC = torch.full((nc, m), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
    assert H.hm_tc_cgemm(dA, dB, dC) == H.HM_OK
    return dC.cpu().numpy().T


@pytest.mark.parametrize("m,k,nc", [(1, 1, 1), (5, 3, 2), (8, 8, 8), (33, 7, 17), (54, 100, 32), (64, 64, 64),
                                    (64, 1000, 64), (27, 6900, 32), (40, 33, 1)])
def test_tc_product_matches_complex128(m, k, nc):
    rng = np.random.default_rng(m * 1000 + k + nc)
    A, B = _cg(rng, (m, k)), _cg(rng, (k, nc))
    C = _run(A, B)
    ref = A.astype(np.complex128) @ B.astype(np.complex128)
    bound = (16 * 2.0 ** -22 + 8 * k * 2.0 ** -24) * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64))
    assert np.all(np.abs(C - ref) <= bound + 1e-30)
    # FP32 level, far below plain TF32 (about 1e-3 relative)
    assert np.linalg.norm(C - ref) <= 2e-6 * np.sqrt(max(k, 1)) * np.linalg.norm(ref)


def test_tc_zero_contraction_writes_zeros():
    A = np.zeros((7, 0), dtype=np.complex64)
    B = np.zeros((0, 3), dtype=np.complex64)
    m, nc = 7, 3
    dA = torch.zeros(1, dtype=torch.complex64, device="cuda")
    dB = torch.zeros(1, dtype=torch.complex64, device="cuda")
    dC = torch.full((nc, m), complex(1.0, 1.0), dtype=torch.complex64, device="cuda")
    assert H.load().hm_tc_cgemm(m, 0, nc, dA.data_ptr(), m, dB.data_ptr(), 1, dC.data_ptr(), m, None) == H.HM_OK
    assert np.all(dC.cpu().numpy() == 0)
    del A, B


def test_tc_columns_independent_of_width():
    rng = np.random.default_rng(5)
    A, B = _cg(rng, (54, 230)), _cg(rng, (230, 64))
    C64 = _run(A, B)
    for w in (1, 5, 16, 33):
        Cw = _run(A, B[:, :w])
        assert np.array_equal(Cw, C64[:, :w]), w
    C1 = _run(A, B[:, 40:41])
    assert np.array_equal(C1[:, 0], C64[:, 40])


def test_tc_rejects_bad_sizes():
    L = H.load()
    x = torch.zeros(64 * 64, dtype=torch.complex64, device="cuda")
    p = x.data_ptr()
    assert L.hm_tc_cgemm(65, 4, 4, p, 65, p, 4, p, 65, None) == H.HM_EINVAL
    assert L.hm_tc_cgemm(4, 4, 65, p, 4, p, 4, p, 4, None) == H.HM_EINVAL
    assert L.hm_tc_cgemm(4, 4, 4, p, 3, p, 4, p, 4, None) == H.HM_EINVAL
    assert L.hm_tc_cgemm(4, -1, 4, p, 4, p, 4, p, 4, None) == H.HM_EINVAL
