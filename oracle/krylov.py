"""The transformed, preconditioned system (Eqs. 22-28) and restarted GMRES (Sec. 5).

System.  Z = Z_N + Z_F (Eq. 11).  With Z_N = L D L^T from ``schur.setup`` the scaled
system (Eqs. 22-27) is [D + L^{-1} Z_F L^{-T}] x~ = L^{-1} b with x = L^{-T} x~, and
the paper solves its block-diagonally (left) preconditioned form (Eq. 28)

    A x~ = c,   A = D^{-1} [D + L^{-1} Z_F L^{-T}],   c = D^{-1} L^{-1} b.

The operator is applied in the paper's form: backward sweep, far-field product,
forward sweep, then D x~ + w and the block solve with D.

GMRES(m), as read here (Sec. 5 gives only the tolerance): x~_0 = 0; Arnoldi with
modified Gram-Schmidt; complex Givens rotations with a real cosine,
c = |a|/rho, s = (a/|a|) conj(b)/rho, rho = sqrt(|a|^2 + |b|^2) (a = 0 -> c = 0,
s = 1); stop when |g_{j+1}| <= tol ||c|| (the residual of the preconditioned system,
which is what GMRES minimises); at every restart the true residual c - A x~ is
recomputed; a happy breakdown when h_{j+1,j} <= 1e-14 ||w||.  ``iters`` counts Arnoldi
steps (operator applications inside cycles).
"""
import numpy as np
import scipy.linalg as sla

from . import schur as _schur


class System:
    """Index maps and operators for one problem + factor (new unknown order)."""

    def __init__(self, prob, F):
        self.prob, self.F = prob, F
        lp = prob.leaf_ptr
        cl = np.concatenate([np.arange(lp[t], lp[t + 1]) for t in F.order])   # new pos -> cluster pos
        self.new2cl = cl
        self.new2orig = np.asarray(prob.perm)[cl]
        self.off = np.concatenate([[0], np.cumsum(F.size)])
        self.n = int(self.off[-1])

    # -- layout helpers ---------------------------------------------------------
    def split(self, x):
        return [x[self.off[k]:self.off[k + 1]].copy() for k in range(self.F.nb)]

    def join(self, v):
        return np.concatenate(v)

    def to_new(self, x_orig):
        return x_orig[self.new2orig]

    def to_orig(self, x_new):
        out = np.empty_like(x_new)
        out[self.new2orig] = x_new
        return out

    # -- Z_F (Eq. 11, far part), in cluster order ---------------------------------
    def far_cluster(self, u):
        p = self.prob
        v = np.zeros(u.shape, dtype=np.complex128)
        for b in range(len(p.far_rank)):
            r0, r1, c0, c1, r = p.far_r0[b], p.far_r1[b], p.far_c0[b], p.far_c1[b], p.far_rank[b]
            m, n = r1 - r0, c1 - c0
            if r < 0:
                B = p.far_U[p.far_uoff[b]:p.far_uoff[b] + m * n].reshape(n, m).T
                v[r0:r1] += B @ u[c0:c1]
                v[c0:c1] += B.T @ u[r0:r1]
            else:
                U = p.far_U[p.far_uoff[b]:p.far_uoff[b] + m * r].reshape(r, m).T
                V = p.far_V[p.far_voff[b]:p.far_voff[b] + n * r].reshape(r, n).T
                v[r0:r1] += U @ (V.T @ u[c0:c1])
                v[c0:c1] += V @ (U.T @ u[r0:r1])
        return v

    def far_new(self, x):
        u = np.zeros(x.shape, dtype=np.complex128)
        u[self.new2cl] = x
        return self.far_cluster(u)[self.new2cl]

    def near_cluster(self, u):
        """Z_N u with the original near blocks (cluster order)."""
        p = self.prob
        lp = p.leaf_ptr
        v = np.zeros(u.shape, dtype=np.complex128)
        for b in range(len(p.near_t)):
            t, s = p.near_t[b], p.near_s[b]
            m, n = lp[t + 1] - lp[t], lp[s + 1] - lp[s]
            B = p.near_data[p.near_off[b]:p.near_off[b] + m * n].reshape(n, m).T
            v[lp[t]:lp[t + 1]] += B @ u[lp[s]:lp[s + 1]]
            if t != s:
                v[lp[s]:lp[s + 1]] += B.T @ u[lp[t]:lp[t + 1]]
        return v

    def Z_new(self, x):
        """Z x in the new (block) order: near blocks as stored plus the far factors."""
        u = np.zeros(x.shape, dtype=np.complex128)
        u[self.new2cl] = x
        return (self.near_cluster(u) + self.far_cluster(u))[self.new2cl]

    def Z_orig(self, x_orig):
        """Z x in the original RWG order (near blocks + far factors)."""
        perm = np.asarray(self.prob.perm)
        u = x_orig[perm]
        v = self.near_cluster(u) + self.far_cluster(u)
        out = np.empty_like(v)
        out[perm] = v
        return out

    # -- Eq. 28 -----------------------------------------------------------------
    def D_mul(self, x):
        v = self.split(x)
        return self.join([self.F.D[k] @ v[k] for k in range(self.F.nb)])

    def D_solve(self, x):
        v = self.split(x)
        return self.join([sla.lu_solve(self.F.lu[k], v[k]) for k in range(self.F.nb)])

    def L_inv(self, x):
        return self.join(_schur.sweep_forward(self.F, self.split(x)))

    def LT_inv(self, x):
        return self.join(_schur.sweep_backward(self.F, self.split(x)))

    def apply_A(self, x):
        """A x~ = D^{-1} [D x~ + L^{-1} Z_F L^{-T} x~]  (Eq. 28)."""
        w = self.L_inv(self.far_new(self.LT_inv(x)))
        return self.D_solve(self.D_mul(x) + w)

    def rhs(self, b_orig):
        """c = D^{-1} L^{-1} b (Eqs. 23, 28), b in original order."""
        return self.D_solve(self.L_inv(self.to_new(b_orig)))

    def solution(self, xt):
        """x = L^{-T} x~ (Eq. 24), returned in original order."""
        return self.to_orig(self.LT_inv(xt))


class _Blocks:
    """Order and sizes of the leaf blocks (what System needs of a factor)."""

    def __init__(self, prob, order):
        self.order = np.asarray(order)
        self.size = np.array([prob.leaf_ptr[t + 1] - prob.leaf_ptr[t] for t in self.order], dtype=np.int64)
        self.nb = len(self.order)


class BlockJacobi(System):
    """The block-diagonal preconditioner of the near-field diagonal blocks, M = diag(Z_kk),
    the low-setup-cost comparison the paper names in Sec. 1 beside the null-field scaling:
    GMRES on M^{-1} Z x = M^{-1} b (left preconditioned, the same GMRES as for Eq. 28), with
    the blocks in the given leaf order and no transformation (x~ = x).  Z x is the H-matrix
    product: near blocks as stored plus the far factors."""

    def __init__(self, prob, order):
        F = _Blocks(prob, order)
        super().__init__(prob, F)
        lp = prob.leaf_ptr
        self.M = []
        for t in F.order:
            b = int(np.nonzero((prob.near_t == t) & (prob.near_s == t))[0][0])
            m = lp[t + 1] - lp[t]
            blk = prob.near_data[prob.near_off[b]:prob.near_off[b] + m * m].reshape(m, m).T
            self.M.append(blk.copy())
        self.lu = [sla.lu_factor(B) for B in self.M]

    def M_solve(self, x):
        v = self.split(x)
        return self.join([sla.lu_solve(self.lu[k], v[k]) for k in range(self.F.nb)])

    def apply_A(self, x):
        return self.M_solve(self.Z_new(x))

    def rhs(self, b_orig):
        return self.M_solve(self.to_new(b_orig))

    def solution(self, xt):
        return self.to_orig(xt)


class NullField(System):
    """The null-field comparison preconditioner, as read here (Sec. 3: the near field scaled
    to diagonal blocks from one side, the fill-in blocks ignored): the elimination of
    ``schur.setup`` restricted to the near-field pattern (``drop_fill``), M = L D L^T, and
    GMRES on M^{-1} Z x = M^{-1} b with M^{-1} = L^{-T} D^{-1} L^{-1} (left preconditioned,
    the same GMRES as for Eq. 28, x~ = x)."""

    def __init__(self, prob, order):
        super().__init__(prob, _schur.setup(prob, order, fill_tol=0.0, drop_fill=True))

    def M_solve(self, x):
        return self.LT_inv(self.D_solve(self.L_inv(x)))

    def apply_A(self, x):
        return self.M_solve(self.Z_new(x))

    def rhs(self, b_orig):
        return self.M_solve(self.to_new(b_orig))

    def solution(self, xt):
        return self.to_orig(xt)


def givens(a, b):
    """(c, s, rho) with [c s; -conj(s) c] [a; b] = [rho; 0], c real."""
    if a == 0:
        return 0.0, 1.0 + 0j, b
    aa, bb = abs(a), abs(b)
    rho_abs = np.hypot(aa, bb)
    c = aa / rho_abs
    s = (a / aa) * np.conj(b) / rho_abs
    rho = (a / aa) * rho_abs
    return c, s, rho


def gmres(apply, c, tol, m, maxit=5000, x0=None, hist=None):
    """Restarted GMRES(m) on A x = c.  Returns (x, iters, relres, converged)."""
    n = c.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else x0.copy()
    cn = np.linalg.norm(c)
    if cn == 0:
        return x, 0, 0.0, True
    it = 0
    while True:
        r = c - apply(x) if it > 0 or x0 is not None else c.copy()
        beta = np.linalg.norm(r)
        if beta <= tol * cn:
            return x, it, beta / cn, True
        if it >= maxit:
            return x, it, beta / cn, False
        Vb = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Vb[0] = r / beta
        j_end = 0
        conv = False
        for j in range(m):
            w = apply(Vb[j])
            it += 1
            wn = np.linalg.norm(w)
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = np.vdot(Vb[i], w)
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = abs(H[j + 1, j]) <= 1e-14 * wn
            if not breakdown:
                Vb[j + 1] = w / H[j + 1, j]
            for i in range(j):                          # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j], rho = givens(H[j, j], H[j + 1, j])
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            j_end = j + 1
            if hist is not None:
                hist.append(abs(g[j + 1]) / cn)
            if abs(g[j + 1]) <= tol * cn or breakdown or it >= maxit:
                conv = abs(g[j + 1]) <= tol * cn or breakdown
                break
        y = sla.solve_triangular(H[:j_end, :j_end], g[:j_end])
        x = x + Vb[:j_end].T @ y
        if conv:
            return x, it, abs(g[j_end]) / cn, True
        if it >= maxit:
            return x, it, abs(g[j_end]) / cn, False


def solve(sysm, b_orig, tol=1e-4, restart=30, maxit=5000, hist=None):
    """Full preconditioned solve of Eq. 28 for one RHS in original order.
    Returns (x_orig, iters, relres_preconditioned, converged)."""
    c = sysm.rhs(b_orig)
    xt, it, rr, ok = gmres(sysm.apply_A, c, tol, restart, maxit, hist=hist)
    return sysm.solution(xt), it, rr, ok
