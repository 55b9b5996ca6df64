"""Symmetric near-field Schur-complement preconditioner (Sec. 3.1, 3.2, 3.4).

Notation (blocks numbered 0..nb-1 in the ordering of Algorithm 1, n_k unknowns each):

* A holds the near field Z_N (Eq. 12) and, as elimination proceeds, its Schur
  complements; only blocks A_ij with i >= j are kept, A_ji = A_ij^T (Sec. 3.2: Z_N is
  complex symmetric, so the left coefficients are transposes of the right ones).
* Step k (Eqs. 13-19): D_k = A_kk; the right scaling coefficients are
  alpha_kj = -D_k^{-1} A_kj for j in S_k (Eq. 14); the step-k Schur complement
  (Eq. 19) updates A_ij -= A_ik D_k^{-1} A_kj for i >= j in S_k, the diagonal blocks in
  full.  S_k = the later blocks coupled to k at step k (the symbolic fill).
* After the last step the near field is blockdiag(D_k) (Eqs. 20-21).  With
  W_kj = D_k^{-1} A_kj = -alpha_kj and L the unit block lower triangle with
  L_jk = W_kj^T: alpha'_{nb-2} ... alpha'_0 = L^{-1} and alpha_0 ... alpha_{nb-2} = L^{-T}
  (Eqs. 20, 23, 24), and Z_N = L D L^T.
* Fill-in compression (Sec. 3.4): after the factorisation every W_kj whose block pair
  (k, j) is not a near-field pair is replaced by its truncated SVD with the smallest
  rank r whose singular-value tail has Frobenius norm <= fill_tol * ||W_kj||_F, kept
  dense when r (n_k + n_j) >= n_k n_j.  Reading taken: compression acts on the stored
  coefficients used by the sweeps, not on the blocks that feed later Schur updates.
* Null-field comparison (Sec. 1 and Sec. 5.2 name it; Sec. 3 says it scales the near field
  to diagonal blocks from one side while ignoring the fill-in blocks).  Reading taken: the
  same block elimination restricted to the near-field pattern, every update whose target
  block is not a near-field pair dropped (a block incomplete factorisation with no fill),
  so that Z_N ~ M = L D L^T with M equal to Z_N on every near-field block pair; the
  preconditioner M^{-1} = L^{-T} D^{-1} L^{-1} is applied from the left.
"""
import numpy as np
import scipy.linalg as sla


def symbolic_fill(nb, pairs):
    """S_k for k = 0..nb-1 (Sec. 3.3, the fill of Figs. 3b-7b): eliminating block k
    couples every pair of its later neighbours.  ``pairs`` are (i, j) block pairs in the
    new numbering."""
    adj = [set() for _ in range(nb)]
    for i, j in pairs:
        if i != j:
            adj[i].add(j)
            adj[j].add(i)
    S = []
    for k in range(nb):
        later = sorted(j for j in adj[k] if j > k)
        S.append(later)
        for a in later:
            for b in later:
                if a != b:
                    adj[a].add(b)
    return S


def near_lists(nb, pairs):
    """S_k without fill: the later blocks that are near-field neighbours of k."""
    S = [set() for _ in range(nb)]
    for i, j in pairs:
        if i != j:
            S[min(i, j)].add(max(i, j))
    return [sorted(x) for x in S]


class Factor:
    """Result of the oracle's setup, in the block numbering of the ordering."""
    pass


def near_blocks_in_order(prob, order):
    """Near-field blocks Z_ij (i >= j) keyed in the new block numbering.
    ``order[p]`` = original leaf id at new position p."""
    pos = np.empty(len(order), dtype=np.int64)
    pos[order] = np.arange(len(order))
    lp = prob.leaf_ptr
    A = {}
    for b in range(len(prob.near_t)):
        t, s = int(prob.near_t[b]), int(prob.near_s[b])
        m, n = lp[t + 1] - lp[t], lp[s + 1] - lp[s]
        blk = prob.near_data[prob.near_off[b]:prob.near_off[b] + m * n].reshape(n, m).T
        i, j = int(pos[t]), int(pos[s])
        if i >= j:
            A[(i, j)] = blk.copy()
        else:
            A[(j, i)] = blk.T.copy()
    return A


def setup(prob, order, fill_tol=1e-2, max_steps=None, compress_in_setup=False, drop_fill=False):
    """The preconditioner of Sec. 3 for block order ``order`` (Algorithm 1 output).
    ``max_steps`` stops after that many elimination steps (a timing sample; the factor is
    then incomplete and only its first steps are valid).

    Fill-in compression (Sec. 3.4) has two readings.  Default (after the factorisation):
    every fill-in coefficient block is truncated once the elimination is complete, and only
    the sweeps use the truncations.  ``compress_in_setup`` (the abstract's reading: the fill-in
    blocks are compressed while the preconditioner is being computed): at elimination step k the fill-in blocks
    W_kj of the new panel are truncated as soon as they are formed, and the Schur updates of
    that step (and so every later pivot block and panel) use the truncations.

    ``drop_fill`` (the null-field reading): S_k = the later near-field neighbours of k, and an
    update A_ij -= A_ik W_kj whose target (i, j) is not a near-field pair is not made."""
    nb = len(order)
    size = np.array([prob.leaf_ptr[order[p] + 1] - prob.leaf_ptr[order[p]] for p in range(nb)], dtype=np.int64)
    A = near_blocks_in_order(prob, order)
    near_pairs = set(A.keys())
    S = near_lists(nb, list(A.keys())) if drop_fill else symbolic_fill(nb, list(A.keys()))
    F = Factor()
    F.order, F.size, F.S, F.nb = np.asarray(order), size, S, nb
    F.near_pairs = near_pairs
    F.D = []
    F.lu = []
    F.W = {}
    for k in range(nb if max_steps is None else min(nb, max_steps)):
        Dk = A.pop((k, k))
        lu = sla.lu_factor(Dk)
        F.D.append(Dk)
        F.lu.append(lu)
        Wk = {j: sla.lu_solve(lu, A[(j, k)].T) for j in S[k]}      # W_kj = D_k^{-1} A_kj
        if compress_in_setup and fill_tol > 0:
            for j in S[k]:
                if (j, k) not in near_pairs:
                    Wk[j] = compress_block(Wk[j], fill_tol)[0]
        for ii, i in enumerate(S[k]):
            Aik = A[(i, k)]
            for j in S[k][:ii + 1]:                                 # i >= j
                upd = Aik @ Wk[j]
                if (i, j) in A:
                    A[(i, j)] = A[(i, j)] - upd
                elif not drop_fill:
                    A[(i, j)] = -upd
        for j in S[k]:
            del A[(j, k)]
            F.W[(k, j)] = Wk[j]
    F.fill_tol = fill_tol
    F.Wc = {}
    F.rank = {}
    for (k, j), W in F.W.items():
        if fill_tol > 0 and (j, k) not in near_pairs:
            F.Wc[(k, j)], F.rank[(k, j)] = compress_block(W, fill_tol)
        else:
            F.Wc[(k, j)] = W
    return F


def compress_block(W, tol):
    """Truncated SVD of Sec. 3.4: returns (approximation, rank) with rank -1 = dense."""
    X, s, Yh = np.linalg.svd(W, full_matrices=False)
    tot = np.sqrt(np.sum(s * s))
    r = len(s)
    for i in range(len(s) + 1):
        tail = np.sqrt(np.sum(s[i:] ** 2))
        if tail <= tol * tot:
            r = i
            break
    m, n = W.shape
    if r * (m + n) >= m * n:
        return W, -1
    return (X[:, :r] * s[:r]) @ Yh[:r, :], r


def sweep_forward(F, v, W=None):
    """v <- L^{-1} v  (the left scalings alpha'_0 .. alpha'_{nb-2} of Eq. 23), in place
    on a list of per-block vectors/panels."""
    W = F.Wc if W is None else W
    for k in range(F.nb):
        for j in F.S[k]:
            v[j] = v[j] - W[(k, j)].T @ v[k]
    return v


def sweep_backward(F, v, W=None):
    """v <- L^{-T} v  (the right scalings alpha_0 .. alpha_{nb-2} of Eq. 24)."""
    W = F.Wc if W is None else W
    for k in range(F.nb - 1, -1, -1):
        for j in F.S[k]:
            v[k] = v[k] - W[(k, j)] @ v[j]
    return v


def ldlt_dense(F, W=None):
    """Dense L D L^T in the new unknown order (small problems only)."""
    W = F.Wc if W is None else W
    off = np.concatenate([[0], np.cumsum(F.size)])
    n = off[-1]
    L = np.eye(n, dtype=np.complex128)
    D = np.zeros((n, n), dtype=np.complex128)
    for k in range(F.nb):
        D[off[k]:off[k + 1], off[k]:off[k + 1]] = F.D[k]
        for j in F.S[k]:
            L[off[j]:off[j + 1], off[k]:off[k + 1]] = W[(k, j)].T
    return L, D


def nnz_coefficients(F):
    """Stored entries of the combined coefficient matrix (Tables 4/6 count): dense W
    blocks n_k n_j, compressed ones r (n_k + n_j), plus the identity diagonal."""
    tot = int(np.sum(F.size))
    for (k, j), W in F.W.items():
        r = F.rank.get((k, j), -1)
        tot += W.size if r < 0 else r * (F.size[k] + F.size[j])
    return tot
