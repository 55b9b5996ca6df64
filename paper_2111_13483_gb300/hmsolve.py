"""Python binding of libhmsolve (include/hmsolve.h): argument marshalling only.

Every function keeps its C name.  Host arrays are numpy; device arrays are torch CUDA
tensors (PyTorch provides device memory and streams, nothing else).  Device vectors are
passed as tensors of shape (nrhs, n), complex128, contiguous: row j is column j of the
column-major n x nrhs matrix the library sees (ld = n).

The library is required: importing this module without a built libhmsolve.so raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

HM_OK, HM_EINVAL, HM_ENOMEM, HM_ESINGULAR, HM_ENOCONV, HM_ETIMEOUT, HM_ECUDA, HM_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
HM_EBUSY = -8
_NAMES = {0: "HM_OK", -1: "HM_EINVAL", -2: "HM_ENOMEM", -3: "HM_ESINGULAR", -4: "HM_ENOCONV", -5: "HM_ETIMEOUT",
          -6: "HM_ECUDA", -7: "HM_ESTATE", -8: "HM_EBUSY"}

OP_A, OP_LINV, OP_LTINV, OP_ZF, OP_DINV, OP_Z = 0, 1, 2, 3, 4, 5
OP32 = 8   # OP32 + op (op 0-4): the complex-FP32 operator of a precision 1 handle

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


class HMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_NAMES.get(code, code), msg))
        self.code = code


class hm_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_leaves", ctypes.c_int32), ("perm", _i32p), ("leaf_ptr", _i32p),
                ("n_near", ctypes.c_int32), ("near_t", _i32p), ("near_s", _i32p), ("near_off", _i64p),
                ("near_data", ctypes.c_void_p), ("near_len", ctypes.c_int64), ("n_far", ctypes.c_int32),
                ("far_r0", _i32p), ("far_r1", _i32p), ("far_c0", _i32p), ("far_c1", _i32p), ("far_rank", _i32p),
                ("far_uoff", _i64p), ("far_voff", _i64p), ("far_U", ctypes.c_void_p), ("far_V", ctypes.c_void_p),
                ("far_U_len", ctypes.c_int64), ("far_V_len", ctypes.c_int64)]


class hm_opts(ctypes.Structure):
    _fields_ = [("ordering", ctypes.c_int32), ("fill_tol", ctypes.c_double), ("precision", ctypes.c_int32),
                ("device", ctypes.c_int32), ("hbm_budget", ctypes.c_size_t), ("stream", ctypes.c_void_p),
                ("preconditioner", ctypes.c_int32), ("compress_in_setup", ctypes.c_int32)]


class hm_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_blocks", ctypes.c_int32), ("near_entries", ctypes.c_int64),
                ("far_entries", ctypes.c_int64), ("fill_blocks", ctypes.c_int64), ("coef_entries", ctypes.c_int64),
                ("coef_entries_dense", ctypes.c_int64), ("diag_entries", ctypes.c_int64),
                ("bandwidth", ctypes.c_int32), ("setup_ms", ctypes.c_double), ("setup_gflop", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t)]


EXPORTS = ["hm_default_opts", "hmat_create", "precond_setup", "solve", "solve_device", "hmat_stats",
           "hm_last_error", "hmat_destroy", "hm_get_order", "hm_get_fill", "hm_get_block", "hm_apply",
           "hm_get_index_map", "hm_plan_order", "hm_plan_fill", "hm_profile", "hm_get_profile",
           "hm_far_apply_noalloc", "hm_get_fill_ranks", "hm_batch_bytes", "hm_batch_open", "hm_batch_submit",
           "hm_batch_step", "hm_batch_result", "hm_batch_close", "hm_set_sweep_schedule",
           "hm_get_profile_cols", "hm_plan_far", "hm_test_hold", "hm_tc_cgemm", "hm_plan_order_method",
           "hm_set_far_schedule", "hm_efie_fill", "hm_efie_far", "hm_set_update_schedule",
           "hm_set_pivot_schedule", "hm_plan_fill_closure"]

KCLASS = ["scatter", "pivot", "panel", "update", "sweep_fwd", "sweep_bwd", "far1", "far2", "diag", "permute",
          "near", "dots", "vec", "small", "compress"]

_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Loads libhmsolve.so (building it in place first if asked); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libhmsolve.so is not built (run __graft_entry__.build())")
    L = ctypes.CDLL(_build.LIB)
    vp = ctypes.c_void_p
    L.hm_default_opts.argtypes = [ctypes.POINTER(hm_opts)]
    L.hmat_create.argtypes = [ctypes.POINTER(hm_desc), ctypes.POINTER(hm_opts), ctypes.POINTER(vp)]
    L.precond_setup.argtypes = [vp]
    L.solve.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                        vp, ctypes.c_int64, _i32p, _f64p]
    L.solve_device.argtypes = L.solve.argtypes
    L.hmat_stats.argtypes = [vp, ctypes.POINTER(hm_stats)]
    L.hm_last_error.argtypes = [vp]
    L.hm_last_error.restype = ctypes.c_char_p
    L.hmat_destroy.argtypes = [vp]
    L.hmat_destroy.restype = None
    L.hm_get_order.argtypes = [vp, _i32p]
    L.hm_get_index_map.argtypes = [vp, _i32p]
    L.hm_get_fill.argtypes = [vp, _i32p, _i32p]
    L.hm_get_block.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp]
    L.hm_apply.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.c_int32]
    L.hm_plan_order.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i32p]
    L.hm_plan_order_method.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i32p]
    L.hm_plan_fill.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, ctypes.c_int64]
    L.hm_plan_fill_closure.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i32p, _i32p,
                                       ctypes.c_int64]
    L.hm_plan_far.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, _i32p,
                              _i64p, _i64p, ctypes.c_int32, _i64p, _i64p]
    L.hm_profile.argtypes = [vp, ctypes.c_int32]
    L.hm_get_profile.argtypes = [vp, ctypes.c_int32, _i64p, _i64p, _f64p]
    L.hm_far_apply_noalloc.argtypes = [vp, vp, vp, ctypes.c_int32]
    L.hm_get_fill_ranks.argtypes = [vp, _i32p]
    L.hm_batch_bytes.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, _i64p]
    L.hm_batch_open.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(vp)]
    L.hm_batch_submit.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int32, _i32p]
    L.hm_batch_step.argtypes = [vp, _i32p, _i32p, _i32p]
    L.hm_batch_result.argtypes = [vp, ctypes.c_int32, vp, _i32p, _f64p]
    L.hm_batch_close.argtypes = [vp]
    L.hm_set_sweep_schedule.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.hm_get_profile_cols.argtypes = [vp, ctypes.c_int32, _i64p]
    L.hm_test_hold.argtypes = [vp, ctypes.c_int32, ctypes.c_int64]
    L.hm_set_far_schedule.argtypes = [vp, ctypes.c_int32]
    L.hm_set_update_schedule.argtypes = [vp, ctypes.c_int32]
    L.hm_set_pivot_schedule.argtypes = [vp, ctypes.c_int32]
    L.hm_tc_cgemm.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_int64, vp, ctypes.c_int64,
                              vp, ctypes.c_int64, vp]
    mesh = [ctypes.c_int32, _f64p, ctypes.c_int32, _i32p, ctypes.c_int32, _i32p, _i32p, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32, _i64p, _i32p, _i64p, _i32p]
    L.hm_efie_fill.argtypes = mesh + [ctypes.c_int32, _i64p, vp, ctypes.c_int64, ctypes.c_int32]
    L.hm_efie_far.argtypes = mesh + [ctypes.c_double, _i32p, _i64p, _i64p, ctypes.c_int64, vp, ctypes.c_int64, vp,
                                     _i64p, ctypes.c_int64, ctypes.c_int32]
    _lib = L
    return L


def _p(a, t):
    return a.ctypes.data_as(t)


class Handle:
    """Owns an hm_handle; destroyed with the object (or explicitly by hmat_destroy)."""

    def __init__(self, ptr, keep):
        self.ptr = ptr
        self._keep = keep
        self.n = keep["n"]
        self.n_leaves = keep["nl"]

    def __del__(self):
        try:
            hmat_destroy(self)
        except Exception:
            pass

    def check(self, code, what):
        if code != HM_OK:
            raise HMError(code, "%s: %s" % (what, hm_last_error(self)))


def hmat_create(prob, ordering=1, fill_tol=0.0, precision=0, device=0, hbm_budget=0, stream=None, preconditioner=0,
                compress_in_setup=0):
    """``prob`` provides perm, leaf_ptr, near_t/near_s/near_off/near_data and
    far_r0/far_r1/far_c0/far_c1/far_rank/far_uoff/far_voff/far_U/far_V (numpy)."""
    L = load()
    k = {}
    k["perm"] = np.ascontiguousarray(prob.perm, dtype=np.int32)
    k["leaf_ptr"] = np.ascontiguousarray(prob.leaf_ptr, dtype=np.int32)
    for f in ("near_t", "near_s", "far_r0", "far_r1", "far_c0", "far_c1", "far_rank"):
        k[f] = np.ascontiguousarray(getattr(prob, f), dtype=np.int32)
    for f in ("near_off", "far_uoff", "far_voff"):
        k[f] = np.ascontiguousarray(getattr(prob, f), dtype=np.int64)
    for f in ("near_data", "far_U", "far_V"):
        k[f] = np.ascontiguousarray(getattr(prob, f), dtype=np.complex128)
    n = len(k["perm"])
    nl = len(k["leaf_ptr"]) - 1
    d = hm_desc()
    d.n, d.n_leaves = n, nl
    d.perm, d.leaf_ptr = _p(k["perm"], _i32p), _p(k["leaf_ptr"], _i32p)
    d.n_near = len(k["near_t"])
    d.near_t, d.near_s, d.near_off = _p(k["near_t"], _i32p), _p(k["near_s"], _i32p), _p(k["near_off"], _i64p)
    d.near_data, d.near_len = k["near_data"].ctypes.data, len(k["near_data"])
    d.n_far = len(k["far_rank"])
    d.far_r0, d.far_r1 = _p(k["far_r0"], _i32p), _p(k["far_r1"], _i32p)
    d.far_c0, d.far_c1 = _p(k["far_c0"], _i32p), _p(k["far_c1"], _i32p)
    d.far_rank = _p(k["far_rank"], _i32p)
    d.far_uoff, d.far_voff = _p(k["far_uoff"], _i64p), _p(k["far_voff"], _i64p)
    d.far_U, d.far_U_len = k["far_U"].ctypes.data, len(k["far_U"])
    d.far_V, d.far_V_len = (k["far_V"].ctypes.data if len(k["far_V"]) else None), len(k["far_V"])
    o = hm_opts()
    L.hm_default_opts(ctypes.byref(o))
    o.ordering, o.fill_tol, o.precision, o.device, o.hbm_budget = ordering, fill_tol, precision, device, hbm_budget
    o.stream = stream
    o.preconditioner = preconditioner
    o.compress_in_setup = compress_in_setup
    h = ctypes.c_void_p()
    code = L.hmat_create(ctypes.byref(d), ctypes.byref(o), ctypes.byref(h))
    if code != HM_OK:
        raise HMError(code, "hmat_create failed (details on stderr)")
    return Handle(h, {"n": n, "nl": nl})


def precond_setup(h):
    h.check(load().precond_setup(h.ptr), "precond_setup")


def solve(h, V, tol=1e-4, restart=30, maxit=5000, raise_on_noconv=False):
    """V: complex128 array (n,) or (n, nrhs) in the original RWG order (host).
    Returns (I, iters, relres, status)."""
    V = np.asarray(V, dtype=np.complex128)
    one = V.ndim == 1
    Vf = np.asfortranarray(V.reshape(h.n, -1))
    nrhs = Vf.shape[1]
    I = np.zeros((h.n, nrhs), dtype=np.complex128, order="F")
    iters = np.zeros(nrhs, dtype=np.int32)
    relres = np.zeros(nrhs, dtype=np.float64)
    code = load().solve(h.ptr, Vf.ctypes.data, nrhs, h.n, tol, restart, maxit, I.ctypes.data, h.n,
                        _p(iters, _i32p), _p(relres, _f64p))
    if code not in (HM_OK, HM_ENOCONV) or (raise_on_noconv and code == HM_ENOCONV):
        h.check(code, "solve")
    return (I[:, 0] if one else I), iters, relres, code


def solve_device(h, dV, dI, tol=1e-4, restart=30, maxit=5000):
    """dV, dI: torch complex128 CUDA tensors of shape (nrhs, n), contiguous (original order)."""
    nrhs = dV.shape[0]
    iters = np.zeros(nrhs, dtype=np.int32)
    relres = np.zeros(nrhs, dtype=np.float64)
    code = load().solve_device(h.ptr, dV.data_ptr(), nrhs, h.n, tol, restart, maxit, dI.data_ptr(), h.n,
                               _p(iters, _i32p), _p(relres, _f64p))
    if code not in (HM_OK, HM_ENOCONV):
        h.check(code, "solve_device")
    return iters, relres, code


def hmat_stats(h):
    s = hm_stats()
    h.check(load().hmat_stats(h.ptr, ctypes.byref(s)), "hmat_stats")
    return {f: getattr(s, f) for f, _ in hm_stats._fields_}


def hm_last_error(h):
    r = load().hm_last_error(h.ptr)
    return r.decode() if r else ""


def hmat_destroy(h):
    if getattr(h, "ptr", None):
        load().hmat_destroy(h.ptr)
        h.ptr = None


def hm_get_order(h):
    out = np.zeros(h.n_leaves, dtype=np.int32)
    h.check(load().hm_get_order(h.ptr, _p(out, _i32p)), "hm_get_order")
    return out


def hm_get_index_map(h):
    out = np.zeros(h.n, dtype=np.int32)
    h.check(load().hm_get_index_map(h.ptr, _p(out, _i32p)), "hm_get_index_map")
    return out


def hm_get_fill(h):
    ptr = np.zeros(h.n_leaves + 1, dtype=np.int32)
    L = load()
    h.check(L.hm_get_fill(h.ptr, _p(ptr, _i32p), None), "hm_get_fill")
    idx = np.zeros(int(ptr[-1]), dtype=np.int32)
    h.check(L.hm_get_fill(h.ptr, _p(ptr, _i32p), _p(idx, _i32p)), "hm_get_fill")
    return ptr, idx


def hm_get_block(h, what, k, shape):
    """Factor block ``what`` (0 D_k, 1 D_k^{-1}, 2 W_k, 3 compressed W_k) of block k,
    returned as a (rows, cols) array; ``shape`` = (rows, cols) expected."""
    out = np.zeros(shape[0] * shape[1], dtype=np.complex128)
    h.check(load().hm_get_block(h.ptr, what, k, out.ctypes.data), "hm_get_block")
    return out.reshape(shape[1], shape[0]).T


def hm_apply(h, op, dx, dy):
    """dx, dy: torch complex128 CUDA tensors (nrhs, n); solve order except op 5 (original)."""
    h.check(load().hm_apply(h.ptr, op, dx.data_ptr(), dy.data_ptr(), dx.shape[0]), "hm_apply")


def hm_plan_order(n_leaves, t, s):
    """Host-only Algorithm 1 ordering (no GPU): order[p] = leaf at position p."""
    t = np.ascontiguousarray(t, dtype=np.int32)
    s = np.ascontiguousarray(s, dtype=np.int32)
    out = np.zeros(n_leaves, dtype=np.int32)
    code = load().hm_plan_order(n_leaves, len(t), _p(t, _i32p), _p(s, _i32p), _p(out, _i32p))
    if code != HM_OK:
        raise HMError(code, "hm_plan_order")
    return out


def hm_plan_order_method(method, n_leaves, t, s):
    """Host-only Algorithm 1 ordering with a chosen method (0 identity, 1 RCM, 2 Sloan)."""
    t = np.ascontiguousarray(t, dtype=np.int32)
    s = np.ascontiguousarray(s, dtype=np.int32)
    out = np.zeros(n_leaves, dtype=np.int32)
    code = load().hm_plan_order_method(method, n_leaves, len(t), _p(t, _i32p), _p(s, _i32p), _p(out, _i32p))
    if code != HM_OK:
        raise HMError(code, "hm_plan_order_method")
    return out


def hm_plan_fill(n_blocks, i, j, closure=1):
    """Host-only S_k lists (no GPU): closure 1 = the symbolic fill, 0 = no fill (the later
    near-field neighbours, the null-field lists).  Returns [S_0, S_1, ...] as lists."""
    i = np.ascontiguousarray(i, dtype=np.int32)
    j = np.ascontiguousarray(j, dtype=np.int32)
    ptr = np.zeros(n_blocks + 1, dtype=np.int32)
    L = load()
    code = L.hm_plan_fill_closure(closure, n_blocks, len(i), _p(i, _i32p), _p(j, _i32p), _p(ptr, _i32p), None, 0)
    if code != HM_OK:
        raise HMError(code, "hm_plan_fill")
    idx = np.zeros(max(1, int(ptr[-1])), dtype=np.int32)
    code = L.hm_plan_fill_closure(closure, n_blocks, len(i), _p(i, _i32p), _p(j, _i32p), _p(ptr, _i32p),
                                  _p(idx, _i32p), len(idx))
    if code != HM_OK:
        raise HMError(code, "hm_plan_fill")
    return [idx[ptr[k]:ptr[k + 1]].tolist() for k in range(n_blocks)]



def hm_plan_far(P):
    """Host-only far-field plan of a problem description (no GPU), as numpy int64 tables:
    seg_ptr, segs (foff, yrow, fi, fk, len, src), part_ptr, tasks (lo, hi, item0, item1),
    items (off, ld, rank, row, isv); see hm_plan_far in the header."""
    L = load()
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    i64 = lambda a: np.ascontiguousarray(a, dtype=np.int64)
    args = [i32(P.leaf_ptr), i32(P.far_r0), i32(P.far_r1), i32(P.far_c0), i32(P.far_c1), i32(P.far_rank),
            i64(P.far_uoff), i64(P.far_voff)]
    lp, r0, r1, c0, c1, rk, uo, vo = args
    widths = {0: 1, 1: 6, 2: 1, 3: 4, 4: 5}
    names = {0: "seg_ptr", 1: "segs", 2: "part_ptr", 3: "tasks", 4: "items"}
    out = {}
    for what, w in widths.items():
        cnt = np.zeros(1, dtype=np.int64)
        call = lambda buf: L.hm_plan_far(int(P.n), len(lp) - 1, _p(lp, _i32p), len(r0), _p(r0, _i32p), _p(r1, _i32p),
                                         _p(c0, _i32p), _p(c1, _i32p), _p(rk, _i32p), _p(uo, _i64p), _p(vo, _i64p),
                                         what, buf, _p(cnt, _i64p))
        code = call(None)
        if code != HM_OK:
            raise HMError(code, "hm_plan_far")
        tab = np.zeros(max(1, int(cnt[0])), dtype=np.int64)
        code = call(_p(tab, _i64p))
        if code != HM_OK:
            raise HMError(code, "hm_plan_far")
        out[names[what]] = tab[:int(cnt[0])].reshape(-1, w) if w > 1 else tab[:int(cnt[0])]
    return out

def hm_profile(h, mode):
    """mode 1: time every launch with CUDA events; 0: stop timing; 2: zero the counters."""
    h.check(load().hm_profile(h.ptr, mode), "hm_profile")


def hm_get_profile(h):
    """{class name: (launches, timed launches, device ms, right-hand-side columns)} per kernel class."""
    out = {}
    L = load()
    for c, name in enumerate(KCLASS):
        a, b, ms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        h.check(L.hm_get_profile(h.ptr, c, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms)), "hm_get_profile")
        cols = ctypes.c_int64()
        h.check(L.hm_get_profile_cols(h.ptr, c, ctypes.byref(cols)), "hm_get_profile_cols")
        out[name] = (a.value, b.value, ms.value, cols.value)
    return out


def hm_far_apply_noalloc(h, dx, dy):
    """y = Z_F x without any device allocation (static library scratch; see the header).
    dx, dy: torch complex128 CUDA tensors (nrhs, n) in solve order.  Returns the status code
    (HM_EINVAL when the call needs more scratch than the static array holds)."""
    return load().hm_far_apply_noalloc(h.ptr, dx.data_ptr(), dy.data_ptr(), dx.shape[0])


def hm_set_sweep_schedule(h, groups=0, kind=0, tile=0):
    """Pins the sweep schedule (column groups 1/2/4; kind 1 row per CTA, 2 two rows, 3 chain +
    helpers, 4 tensor cores, 5 / 6 clusters of 8 / 16 CTAs; tile shape 0-2 of kind 1); (0, 0) =
    tuned."""
    h.check(load().hm_set_sweep_schedule(h.ptr, groups, kind, tile), "hm_set_sweep_schedule")


def hm_test_hold(h, block=-1, wait_ns=0):
    """Test hook: the sweeps leave block row ``block`` (solve order) out and every device-side
    wait gives up after ``wait_ns`` (0 = the default 2 s); (-1, 0) restores normal operation."""
    h.check(load().hm_test_hold(h.ptr, block, wait_ns), "hm_test_hold")


def hm_tc_cgemm(dA, dB, dC, stream=None):
    """C = A B on the tensor-core micro-kernel of the complex-FP32 sweeps.  Torch complex64
    CUDA tensors, contiguous: dA (k, m), dB (ncols, k), dC (ncols, m) -- row j of each is column
    j of the column-major matrix the library sees.  Returns the status code."""
    k, m = dA.shape
    nc = dB.shape[0]
    return load().hm_tc_cgemm(m, k, nc, dA.data_ptr(), m, dB.data_ptr(), k, dC.data_ptr(), m, stream)


def hm_set_far_schedule(h, kind=0):
    """Complex-FP32 far-field products: 1 CUDA cores, 2 tensor cores, 0 default (1)."""
    h.check(load().hm_set_far_schedule(h.ptr, kind), "hm_set_far_schedule")


def hm_set_update_schedule(h, kind=0):
    """Complex-FP32 Schur updates of precond_setup: 1 CUDA cores, 2 tensor cores, 0 default (1)."""
    h.check(load().hm_set_update_schedule(h.ptr, kind), "hm_set_update_schedule")


def hm_set_pivot_schedule(h, ctas=0):
    """CTAs per FP64 pivot inversion in precond_setup: 1, or a cluster of 2, 4 or 8 (bitwise
    the same inverses); 0 = the default (8)."""
    h.check(load().hm_set_pivot_schedule(h.ptr, ctas), "hm_set_pivot_schedule")


def hm_get_fill_ranks(h):
    """Sec. 3.4 ranks per S_k entry (hm_get_fill order): r >= 0 compressed, -1 dense."""
    ptr, idx = hm_get_fill(h)
    out = np.zeros(max(1, len(idx)), dtype=np.int32)
    h.check(load().hm_get_fill_ranks(h.ptr, _p(out, _i32p)), "hm_get_fill_ranks")
    return out[:len(idx)]


class Batch:
    """Continuous-batching slot engine over one handle (hm_batch_* in the header).

    ``submit(V)`` places a right-hand side (complex128 (n,), original order; numpy or a torch
    CUDA tensor) in a free slot and returns the slot (None when all are occupied);
    ``step()`` advances every occupied slot by one GMRES step and returns the slots that
    finished; ``result(slot)`` returns (I, iters, relres, status) and frees the slot."""

    def __init__(self, h, slots, restart=30):
        self.h, self.slots, self.restart = h, slots, restart
        p = ctypes.c_void_p()
        h.check(load().hm_batch_open(h.ptr, slots, restart, ctypes.byref(p)), "hm_batch_open")
        self.ptr = p
        self._fin = np.zeros(slots, dtype=np.int32)
        self._keep = {}

    @staticmethod
    def bytes(h, slots, restart=30):
        b = ctypes.c_int64()
        h.check(load().hm_batch_bytes(h.ptr, slots, restart, ctypes.byref(b)), "hm_batch_bytes")
        return b.value

    def submit(self, V, tol=1e-4, maxit=5000):
        if hasattr(V, "data_ptr"):
            ptr, keep = V.data_ptr(), V
        else:
            keep = np.ascontiguousarray(V, dtype=np.complex128)
            ptr = keep.ctypes.data
        slot = ctypes.c_int32()
        code = load().hm_batch_submit(self.ptr, ptr, tol, maxit, ctypes.byref(slot))
        if code == HM_EBUSY:
            return None
        self.h.check(code, "hm_batch_submit")
        return slot.value

    def step(self):
        nf, na = ctypes.c_int32(), ctypes.c_int32()
        self.h.check(load().hm_batch_step(self.ptr, _p(self._fin, _i32p), ctypes.byref(nf), ctypes.byref(na)),
                     "hm_batch_step")
        self.active = na.value
        return self._fin[:nf.value].tolist()

    def result(self, slot, out=None):
        """out: optional torch CUDA complex128 tensor (n,) to receive I on the device."""
        it, rr = ctypes.c_int32(), ctypes.c_double()
        if out is not None:
            code = load().hm_batch_result(self.ptr, slot, out.data_ptr(), ctypes.byref(it), ctypes.byref(rr))
            I = out
        else:
            I = np.zeros(self.h.n, dtype=np.complex128)
            code = load().hm_batch_result(self.ptr, slot, I.ctypes.data, ctypes.byref(it), ctypes.byref(rr))
        if code not in (HM_OK, HM_ENOCONV):
            self.h.check(code, "hm_batch_result")
        return I, it.value, rr.value, code

    def close(self):
        if getattr(self, "ptr", None):
            load().hm_batch_close(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """The mesh arguments of hm_efie_fill / hm_efie_far: vertices, triangles, and per RWG
    function its T+ / T- triangles and their free vertices."""

    def __init__(self, V, T, tri, free, k, eta0, r_abs=0.2, c_rel=3.0):
        self.V = np.ascontiguousarray(V, dtype=np.float64)
        self.T = np.ascontiguousarray(T, dtype=np.int32)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.free = np.ascontiguousarray(free, dtype=np.int32)
        self.k, self.eta0, self.r_abs, self.c_rel = float(k), float(eta0), float(r_abs), float(c_rel)

    def args(self):
        return [len(self.V), _p(self.V, _f64p), len(self.T), _p(self.T, _i32p), len(self.tri), _p(self.tri, _i32p),
                _p(self.free, _i32p), self.k, self.eta0, self.r_abs, self.c_rel]


def _block_lists(rows_list, cols_list):
    rptr = np.zeros(len(rows_list) + 1, dtype=np.int64)
    cptr = np.zeros(len(cols_list) + 1, dtype=np.int64)
    rptr[1:] = np.cumsum([len(r) for r in rows_list])
    cptr[1:] = np.cumsum([len(c) for c in cols_list])
    ridx = np.ascontiguousarray(np.concatenate(rows_list) if len(rows_list) else np.zeros(0), dtype=np.int32)
    cidx = np.ascontiguousarray(np.concatenate(cols_list) if len(cols_list) else np.zeros(0), dtype=np.int32)
    return rptr, ridx, cptr, cidx


def hm_efie_fill(mesh, rows_list, cols_list, mirror=0, device=0, scratch_bytes=0):
    """Dense blocks of Eq. 7 (RWG index lists per block); returns (flat complex128, offsets)."""
    L = load()
    rptr, ridx, cptr, cidx = _block_lists(rows_list, cols_list)
    off = np.zeros(len(rows_list) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) * len(c) for r, c in zip(rows_list, cols_list)])
    out = np.empty(int(off[-1]), dtype=np.complex128)
    code = L.hm_efie_fill(*mesh.args(), len(rows_list), _p(rptr, _i64p), _p(ridx, _i32p), _p(cptr, _i64p),
                          _p(cidx, _i32p), mirror, _p(off, _i64p), out.ctypes.data if len(out) else None,
                          scratch_bytes, device)
    if code != HM_OK:
        raise HMError(code, "hm_efie_fill failed (details on stderr)")
    return out, off


def hm_efie_far(mesh, rows_list, cols_list, eps, device=0, cap=None, scratch_bytes=0):
    """ACA + re-compression of admissible blocks; returns (rank, uoff, voff, U, V) in the
    layout of hm_desc's far field (rank -1: the dense block at U[uoff])."""
    L = load()
    nb = len(rows_list)
    rptr, ridx, cptr, cidx = _block_lists(rows_list, cols_list)
    rank = np.zeros(nb, dtype=np.int32)
    uoff = np.zeros(nb, dtype=np.int64)
    voff = np.zeros(nb, dtype=np.int64)
    need = np.zeros(2, dtype=np.int64)
    if cap is None:
        # every block at its ACA rank cap (only the pages written are ever touched); more is
        # needed only where dense blocks outgrow that, and the call then reports it
        m = np.diff(rptr)
        n = np.diff(cptr)
        cb = np.minimum(np.minimum(np.minimum(m, n), m * n // (m + n) + 1), 256)
        cap = (int(np.sum(np.minimum(m * n, m * cb))), int(np.sum(n * cb)))
    for _ in range(2):
        U = np.empty(max(cap[0], 1), dtype=np.complex128)
        V = np.empty(max(cap[1], 1), dtype=np.complex128)
        code = L.hm_efie_far(*mesh.args(), nb, _p(rptr, _i64p), _p(ridx, _i32p), _p(cptr, _i64p), _p(cidx, _i32p),
                             eps, _p(rank, _i32p), _p(uoff, _i64p), _p(voff, _i64p), cap[0], U.ctypes.data, cap[1],
                             V.ctypes.data, _p(need, _i64p), scratch_bytes, device)
        if code == HM_ENOMEM and (need[0] > cap[0] or need[1] > cap[1]):
            cap = (int(need[0]), int(need[1]))
            continue
        if code != HM_OK:
            raise HMError(code, "hm_efie_far failed (details on stderr)")
        return rank, uoff, voff, U[:need[0]], V[:need[1]]
    raise HMError(HM_ENOMEM, "hm_efie_far: factor storage")
