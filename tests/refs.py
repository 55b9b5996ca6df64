"""Reference constructions shared by GPU parity tests (built from the oracle)."""
import numpy as np

import paper_2111_13483_gb300 as hm


def truncated_at(F, h):
    """The oracle's coefficient blocks truncated (FP64 SVD) at the ranks handle h chose: the
    reference for a complex-FP32 setup, whose Jacobi ranks can differ from the FP64 ones where
    a singular value sits at the cut."""
    ranks = hm.hmsolve.hm_get_fill_ranks(h)
    out, e = {}, 0
    for k in range(F.nb):
        for j in F.S[k]:
            r = int(ranks[e])
            e += 1
            W = F.W[(k, j)]
            if r < 0:
                out[(k, j)] = W
            else:
                X, sv, Yh = np.linalg.svd(W, full_matrices=False)
                out[(k, j)] = (X[:, :r] * sv[:r]) @ Yh[:r, :]
    return out
