"""Seeded H-matrix EFIE problems: the inputs of the preconditioned solve.

``build(spec)`` runs mesh -> RWG -> cluster tree -> partition -> near-field blocks
(Eq. 7, dense) -> far-field ACA + SVD re-compression (Eqs. 9-10) -> plane-wave RHS,
and returns a ``Problem`` laid out the way the solver library ingests it:

* ``perm[i]``: original RWG index of cluster-order position i;
* ``leaf_ptr``: leaf ranges in cluster order;
* near blocks for leaf pairs t <= s, column-major n_t x n_s (the (s, t) block is the
  transpose: Z is complex symmetric);
* far blocks for admissible pairs whose row range precedes the column range, as
  U (m x r) V (n x r)^T, column-major, or as a dense m x n block (rank -1) when
  r (m + n) >= m n.

Re-compression: QR of U and V, SVD of the small core, truncation to the smallest r
whose singular-value tail has Frobenius norm <= eps times the whole (Sec. 2, the
re-compressed ACA the paper builds on).
"""
import ctypes
import hashlib
import os
import pickle
import subprocess
import tempfile
import threading

import numpy as np

from . import mesh as _mesh
from . import tree as _tree

ETA0 = 376.730313668
K0 = 2.0 * np.pi            # wavelength 1
_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_efie.so")
_lock = threading.Lock()
_lib = None


def build_lib(force=False):
    """Compile the C entry/ACA evaluator in place (gcc + OpenMP)."""
    src = os.path.join(_HERE, "csrc", "efie.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build_lib()
            L = ctypes.CDLL(_SO)
            vp, i32p, i64p, f64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
            L.efie_create.restype = vp
            L.efie_create.argtypes = [ctypes.c_int, f64p, ctypes.c_int, i32p, ctypes.c_int, i32p, i32p,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.efie_destroy.argtypes = [vp]
            L.efie_fill_blocks.argtypes = [vp, ctypes.c_int, i64p, i32p, i64p, i32p, i64p, f64p]
            L.efie_aca_blocks.argtypes = [vp, ctypes.c_int, i64p, i32p, i64p, i32p, ctypes.c_double, i32p,
                                          ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), i32p]
            L.efie_free.argtypes = [vp]
            L.efie_potint.argtypes = [f64p, f64p, f64p, f64p, f64p]
            L.efie_rule.argtypes = [f64p, f64p]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def quadrature_rule():
    w = np.zeros(7)
    b = np.zeros(21)
    lib().efie_rule(_p(w, ctypes.c_double), _p(b, ctypes.c_double))
    return w, b.reshape(7, 3)


def potential_integrals(P, r):
    """Closed-form (\\int 1/R, \\int (r'-rho)/R) over triangle P (3x3) at point r."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n = np.ascontiguousarray(n / np.linalg.norm(n))
    r = np.ascontiguousarray(r, dtype=np.float64)
    s0 = np.zeros(1)
    sv = np.zeros(3)
    lib().efie_potint(_p(P, ctypes.c_double), _p(n, ctypes.c_double), _p(r, ctypes.c_double),
                      _p(s0, ctypes.c_double), _p(sv, ctypes.c_double))
    return s0[0], sv


class EntryEvaluator:
    """Z(i, j) of Eq. 7 for sets of RWG indices (original numbering)."""

    def __init__(self, rwg, k=K0, eta0=ETA0, r_abs=0.2, c_rel=3.0):
        self.rwg = rwg
        self.k = k
        self.eta0 = eta0
        L = lib()
        self._V = np.ascontiguousarray(rwg.V, dtype=np.float64)
        self._T = np.ascontiguousarray(rwg.T, dtype=np.int32)
        self._tri = np.ascontiguousarray(rwg.tri, dtype=np.int32)
        self._free = np.ascontiguousarray(rwg.free, dtype=np.int32)
        self.ctx = L.efie_create(len(self._V), _p(self._V, ctypes.c_double), len(self._T), _p(self._T, ctypes.c_int32),
                                 rwg.n, _p(self._tri, ctypes.c_int32), _p(self._free, ctypes.c_int32),
                                 k, eta0, r_abs, c_rel)

    def __del__(self):
        try:
            if self.ctx:
                lib().efie_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    def blocks(self, rows_list, cols_list):
        """Dense blocks; returns one flat complex array and offsets."""
        rptr = np.zeros(len(rows_list) + 1, dtype=np.int64)
        cptr = np.zeros(len(cols_list) + 1, dtype=np.int64)
        rptr[1:] = np.cumsum([len(r) for r in rows_list])
        cptr[1:] = np.cumsum([len(c) for c in cols_list])
        ridx = np.ascontiguousarray(np.concatenate(rows_list) if rows_list else np.zeros(0), dtype=np.int32)
        cidx = np.ascontiguousarray(np.concatenate(cols_list) if cols_list else np.zeros(0), dtype=np.int32)
        sizes = np.array([len(r) * len(c) for r, c in zip(rows_list, cols_list)], dtype=np.int64)
        off = np.zeros(len(sizes) + 1, dtype=np.int64)
        off[1:] = np.cumsum(sizes)
        out = np.zeros(int(off[-1]), dtype=np.complex128)
        if len(rows_list):
            lib().efie_fill_blocks(self.ctx, len(rows_list), _p(rptr, ctypes.c_int64), _p(ridx, ctypes.c_int32),
                                   _p(cptr, ctypes.c_int64), _p(cidx, ctypes.c_int32), _p(off, ctypes.c_int64),
                                   out.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out, off

    def block(self, rows, cols):
        out, _ = self.blocks([np.asarray(rows)], [np.asarray(cols)])
        return out.reshape(len(cols), len(rows)).T

    def dense(self):
        """The full matrix of Eq. 7 (small meshes), filled in column strips in parallel."""
        n = self.rwg.n
        idx = np.arange(n)
        strips = [idx[c:c + 32] for c in range(0, n, 32)]
        out, off = self.blocks([idx] * len(strips), strips)
        Z = np.empty((n, n), dtype=np.complex128)
        for s, cols in enumerate(strips):
            Z[:, cols] = out[off[s]:off[s + 1]].reshape(len(cols), n).T
        return Z

    def aca(self, rows_list, cols_list, eps):
        """ACA factors per block: (U m x r, V n x r) or None when the rank reached
        floor(m n / (m + n)) + 1 (dense storage is then cheaper) without converging."""
        nb = len(rows_list)
        m = np.array([len(r) for r in rows_list], dtype=np.int64)
        n = np.array([len(c) for c in cols_list], dtype=np.int64)
        maxr = np.minimum(np.minimum(m, n), (m * n) // (m + n) + 1).astype(np.int32)
        rptr = np.zeros(nb + 1, dtype=np.int64)
        cptr = np.zeros(nb + 1, dtype=np.int64)
        rptr[1:] = np.cumsum(m)
        cptr[1:] = np.cumsum(n)
        uptr = (ctypes.c_void_p * nb)()
        vptr = (ctypes.c_void_p * nb)()
        rank = np.zeros(nb, dtype=np.int32)
        ridx = np.ascontiguousarray(np.concatenate(rows_list), dtype=np.int32)
        cidx = np.ascontiguousarray(np.concatenate(cols_list), dtype=np.int32)
        L = lib()
        L.efie_aca_blocks(self.ctx, nb, _p(rptr, ctypes.c_int64), _p(ridx, ctypes.c_int32),
                          _p(cptr, ctypes.c_int64), _p(cidx, ctypes.c_int32), eps, _p(maxr, ctypes.c_int32),
                          uptr, vptr, _p(rank, ctypes.c_int32))
        out = []
        for b in range(nb):
            r = int(rank[b])
            if r < 0:
                out.append(None)
                continue
            mb, nbb = int(m[b]), int(n[b])
            if r == 0:
                Ub = np.zeros((mb, 0), np.complex128)
                Vb = np.zeros((nbb, 0), np.complex128)
            else:
                Ub = np.ctypeslib.as_array(ctypes.cast(uptr[b], ctypes.POINTER(ctypes.c_double)),
                                           shape=(r * mb * 2,)).view(np.complex128).reshape(r, mb).T.copy()
                Vb = np.ctypeslib.as_array(ctypes.cast(vptr[b], ctypes.POINTER(ctypes.c_double)),
                                           shape=(r * nbb * 2,)).view(np.complex128).reshape(r, nbb).T.copy()
            L.efie_free(uptr[b])
            L.efie_free(vptr[b])
            out.append((Ub, Vb))
        return out


def recompress(U, V, eps):
    """QR(U), QR(V), SVD of the core, truncated with a relative Frobenius tail <= eps."""
    if U.shape[1] == 0:
        return U, V
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(V)
    X, s, Yh = np.linalg.svd(Ru @ Rv.T)
    tot = np.sqrt(np.sum(s * s))
    tail = np.sqrt(np.maximum(np.cumsum((s * s)[::-1])[::-1], 0.0))   # tail[i] = ||s[i:]||
    r = len(s)
    for i in range(len(s) + 1):
        t = tail[i] if i < len(s) else 0.0
        if t <= eps * tot:
            r = i
            break
    return Qu @ (X[:, :r] * s[:r]), Qv @ Yh[:r, :].T


class Problem:
    """One seeded EFIE H-matrix problem (see module docstring for the layout)."""

    def plane_wave(self, khat, pol):
        """V_m = <f_m, E_inc>, E_inc = pol e^{-j k khat.r}, original RWG order."""
        return plane_wave_rhs(self.rwg, np.asarray(khat, float), np.asarray(pol, float), self.k)

    @property
    def n(self):
        return self.rwg.n

    def stats(self):
        nl = len(self.leaf_ptr) - 1
        near = int(sum((self.leaf_ptr[t + 1] - self.leaf_ptr[t]) * (self.leaf_ptr[s + 1] - self.leaf_ptr[s])
                       for t, s in zip(self.near_t, self.near_s)))
        fr = self.far_rank
        m = self.far_r1 - self.far_r0
        n = self.far_c1 - self.far_c0
        far = int(np.sum(np.where(fr >= 0, fr * (m + n), m * n)))
        return {"n": int(self.n), "n_leaves": int(nl), "n_near": int(len(self.near_t)), "near_entries_half": near,
                "n_far": int(len(fr)), "far_entries_half": far, "n_far_dense": int(np.sum(fr < 0))}


def plane_wave_rhs(rwg, khat, pol, k=K0):
    w, bary = quadrature_rule()
    P = rwg.V[rwg.T]                                    # nt x 3 x 3
    Q = np.einsum("qa,tad->tqd", bary, P)               # nt x 7 x 3
    phase = np.exp(-1j * k * (Q @ khat))                # nt x 7
    out = np.zeros(rwg.n, dtype=np.complex128)
    for s, sign in ((0, 1.0), (1, -1.0)):
        t = rwg.tri[:, s]
        vf = rwg.V[rwg.free[:, s]]
        rho = Q[t] - vf[:, None, :]                     # nb x 7 x 3
        val = np.einsum("q,bq,bq->b", w, rho @ pol, phase[t])
        out += sign * 0.5 * rwg.length * val
    return out


def far_field(rwg, I, rhat, k=K0, eta0=ETA0):
    """F(rhat) = \\int J e^{j k rhat.r'} ds' for J = sum I_n f_n, rows of rhat (M x 3)."""
    w, bary = quadrature_rule()
    P = rwg.V[rwg.T]
    Q = np.einsum("qa,tad->tqd", bary, P)
    F = np.zeros((len(rhat), 3), dtype=np.complex128)
    for s, sign in ((0, 1.0), (1, -1.0)):
        t = rwg.tri[:, s]
        vf = rwg.V[rwg.free[:, s]]
        rho = Q[t] - vf[:, None, :]                     # nb x 7 x 3
        coef = sign * 0.5 * rwg.length * I              # nb
        ph = np.exp(1j * k * np.einsum("bqd,md->mbq", Q[t], rhat))  # M x nb x 7
        F += np.einsum("q,b,mbq,bqd->md", w, coef, ph, rho)
    return F


def bistatic_rcs(rwg, I, rhat, k=K0, eta0=ETA0):
    """sigma(rhat) = (k eta0)^2/(4 pi) |F_perp|^2 for a unit incident field (m^2, lambda = 1)."""
    F = far_field(rwg, I, rhat, k, eta0)
    Fp = F - (np.einsum("md,md->m", F, rhat))[:, None] * rhat
    return (k * eta0) ** 2 / (4.0 * np.pi) * np.sum(np.abs(Fp) ** 2, axis=1)


SPECS = {
    # 1920-unknown sphere: icosphere d=3, radius 0.6 lambda
    "sphere1920": dict(kind="sphere", d=3, a=0.6, leaf=64, eta=1.0, aca_eps=1e-3),
    # 30,720-unknown sphere: icosphere d=5, radius 2.4 lambda
    "sphere30720": dict(kind="sphere", d=5, a=2.4, leaf=64, eta=1.0, aca_eps=1e-3),
    # 10 x 10 lambda jittered plate, 100 x 100 grid (29,800 unknowns)
    "plate29800": dict(kind="plate", n=100, w=10.0, jitter=0.1, seed=0, leaf=64, eta=1.0, aca_eps=1e-3),
    # 122,880-unknown sphere: icosphere d=6, radius 5 lambda, ACA 1e-4
    "sphere122880": dict(kind="sphere", d=6, a=5.0, leaf=64, eta=1.0, aca_eps=1e-4),
    # mid-size sphere (profiling captures, mid-size parity): icosphere d=4, radius 1.2 lambda
    "sphere7680": dict(kind="sphere", d=4, a=1.2, leaf=64, eta=1.0, aca_eps=1e-3),
    # small cases for tests
    "sphere480":dict(kind="sphere", d=2, a=0.3, leaf=32, eta=1.0, aca_eps=1e-3),
    "plate_tiny": dict(kind="plate", n=8, w=0.8, jitter=0.1, seed=0, leaf=16, eta=1.0, aca_eps=1e-3),
    # 2 x 2 lambda jittered plate on the same 0.1 lambda grid as plate29800 (1160 unknowns)
    "plate1160": dict(kind="plate", n=20, w=2.0, jitter=0.1, seed=0, leaf=64, eta=1.0, aca_eps=1e-3),
}


def make_mesh(spec):
    if spec["kind"] == "sphere":
        return _mesh.icosphere(spec["d"], spec["a"])
    if spec["kind"] == "plate":
        return _mesh.plate(spec["n"], spec["w"], spec.get("jitter", 0.1), spec.get("seed", 0))
    raise ValueError(spec["kind"])


def build(spec, cache=True, verbose=False):
    """Build (or load from the temp-dir cache) the problem for a spec dict or name."""
    if isinstance(spec, str):
        spec = SPECS[spec]
    key = hashlib.sha1(repr(sorted(spec.items())).encode() + open(os.path.join(_HERE, "csrc", "efie.c"), "rb").read()
                       + open(__file__, "rb").read() + open(_tree.__file__, "rb").read()
                       + open(_mesh.__file__, "rb").read()).hexdigest()[:16]
    path = os.path.join(tempfile.gettempdir(), "efie_problem_%s.pkl" % key)
    if cache and os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    P = _build(spec, verbose)
    P.spec = dict(spec)
    if cache:
        tmp = path + ".%d" % os.getpid()
        with open(tmp, "wb") as f:
            pickle.dump(P, f, protocol=4)
        os.replace(tmp, path)
    return P


def _build(spec, verbose=False):
    import time
    t0 = time.time()
    V, T = make_mesh(spec)
    rwg = _mesh.RWG(V, T)
    pts = rwg.midpoints()
    root, leaves, perm = _tree.build_tree(pts, spec.get("leaf", 64), vertices=V, fixed_level=spec.get("level"))
    blo, bhi = rwg.support_boxes()
    _tree.attach_boxes(root, perm, blo, bhi)
    near, far = _tree.partition(root, spec.get("eta", 1.0))
    leaf_ptr = np.array([lf.lo for lf in leaves] + [leaves[-1].hi], dtype=np.int64)
    ev = EntryEvaluator(rwg)
    P = Problem()
    P.rwg, P.k, P.eta0 = rwg, ev.k, ev.eta0
    P.perm = perm.astype(np.int32)
    P.leaf_ptr = leaf_ptr.astype(np.int32)
    nr = sorted({(min(t, s), max(t, s)) for t, s in near})
    P.near_t = np.array([a for a, _ in nr], dtype=np.int32)
    P.near_s = np.array([b for _, b in nr], dtype=np.int32)
    rows = [perm[leaf_ptr[t]:leaf_ptr[t + 1]] for t, _ in nr]
    cols = [perm[leaf_ptr[s]:leaf_ptr[s + 1]] for _, s in nr]
    data, off = ev.blocks(rows, cols)
    for b, (t, s) in enumerate(nr):          # diagonal blocks: upper triangle mirrored
        if t == s:
            m = leaf_ptr[t + 1] - leaf_ptr[t]
            blk = data[off[b]:off[b + 1]].reshape(m, m).T
            sym = np.triu(blk) + np.triu(blk, 1).T
            data[off[b]:off[b + 1]] = sym.T.ravel()
    P.near_off = off[:-1].astype(np.int64)
    P.near_data = data
    t1 = time.time()
    fr = [(t, s) for t, s in far if t.lo < s.lo]
    fr.sort(key=lambda ts: (ts[0].lo, ts[1].lo, ts[0].hi, ts[1].hi))
    rl = [perm[t.lo:t.hi] for t, _ in fr]
    cl = [perm[s.lo:s.hi] for _, s in fr]
    eps = spec.get("aca_eps", 1e-3)
    facs = ev.aca(rl, cl, eps) if fr else []
    t2 = time.time()
    ranks, U_parts, V_parts, uoff, voff = [], [], [], [], []
    dense_idx = []
    cu = cv = 0
    for b, ((t, s), f) in enumerate(zip(fr, facs)):
        m, n = t.hi - t.lo, s.hi - s.lo
        if f is not None:
            Ub, Vb = recompress(f[0], f[1], eps)
            r = Ub.shape[1]
            if r * (m + n) < m * n:
                ranks.append(r)
                uoff.append(cu)
                voff.append(cv)
                U_parts.append(np.asfortranarray(Ub).ravel(order="F"))
                V_parts.append(np.asfortranarray(Vb).ravel(order="F"))
                cu += m * r
                cv += n * r
                continue
        ranks.append(-1)
        uoff.append(cu)
        voff.append(cv)
        dense_idx.append(b)
        U_parts.append(None)
        cu += m * n
    if dense_idx:
        dd, doff = ev.blocks([rl[b] for b in dense_idx], [cl[b] for b in dense_idx])
        for j, b in enumerate(dense_idx):
            U_parts[b] = dd[doff[j]:doff[j + 1]]
    P.far_r0 = np.array([t.lo for t, _ in fr], dtype=np.int32)
    P.far_r1 = np.array([t.hi for t, _ in fr], dtype=np.int32)
    P.far_c0 = np.array([s.lo for _, s in fr], dtype=np.int32)
    P.far_c1 = np.array([s.hi for _, s in fr], dtype=np.int32)
    P.far_rank = np.array(ranks, dtype=np.int32)
    P.far_uoff = np.array(uoff, dtype=np.int64)
    P.far_voff = np.array(voff, dtype=np.int64)
    P.far_U = np.concatenate(U_parts) if U_parts else np.zeros(0, np.complex128)
    P.far_V = np.concatenate([v for v in V_parts]) if V_parts else np.zeros(0, np.complex128)
    if verbose:
        print("build: near %.1fs aca %.1fs recompress %.1fs" % (t1 - t0, t2 - t1, time.time() - t2), P.stats())
    return P
