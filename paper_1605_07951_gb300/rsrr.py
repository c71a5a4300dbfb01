"""Thin ctypes binding of include/rsrr.h (same names, argument marshalling only).

Every computation runs in librsrr.so (CUDA, sm_103a).  There is no CPU
fallback: importing this module fails loudly if the library is missing.
Device buffers may be given as torch CUDA tensors (their data_ptr() is
passed) and streams as torch.cuda.Stream objects or raw handles.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsrr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`"
        " (the resolvent-sampling library has no CPU fallback)")

_lib = C.CDLL(LIB_PATH)

# ---------------------------------------------------------------- constants
RSRR_OK, RSRR_EINVAL, RSRR_ENOMEM, RSRR_ESINGULAR = 0, -1, -2, -3
RSRR_ENOCONV, RSRR_ETIMEOUT, RSRR_ECUDA, RSRR_ESTATE, RSRR_WGAP = -4, -5, -6, -7, 1
(RSRR_F_ONE, RSRR_F_ZPOW, RSRR_F_RATIONAL, RSRR_F_INV, RSRR_F_SQRT, RSRR_F_EXP, RSRR_F_TAYLOR,
 RSRR_F_CALLBACK) = range(8)
RSRR_REGION_ELLIPSE, RSRR_REGION_POINTS, RSRR_REGION_INTERVAL, RSRR_REGION_RECT = 0, 1, 2, 3
RSRR_METHOD_RSRR, RSRR_METHOD_SSRR_M, RSRR_METHOD_SS_RI = 0, 1, 2
RSRR_REFINE_IR, RSRR_REFINE_GMRES = 0, 1
RSRR_PREC_FP64, RSRR_PREC_MIXED = 0, 1
RSRR_GEMM_AUTO, RSRR_GEMM_FP64, RSRR_GEMM_OZAKI, RSRR_GEMM_OZAKI_MMA = 0, 1, 2, 3
(RSRR_FLAG_PLAIN_SOLVE, RSRR_FLAG_ONE_CTA_LU, RSRR_FLAG_INJECT_TIMEOUT, RSRR_FLAG_SIMT_DENSE_UPDATE,
 RSRR_FLAG_GRAPH, RSRR_FLAG_AUTOTUNE, RSRR_FLAG_WIDE_SOLVE_ONLY, RSRR_FLAG_REAL,
 RSRR_FLAG_CHUNK_POINTS) = 1, 2, 4, 8, 16, 32, 64, 128, 256
RSRR_NEP_SPARSE, RSRR_NEP_HELMHOLTZ, RSRR_NEP_DENSE = 0, 1, 2
RSRR_MAX_TERMS = 8
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ESINGULAR", -4: "ENOCONV",
                -5: "ETIMEOUT", -6: "ECUDA", -7: "ESTATE", 1: "WGAP"}


# ---------------------------------------------------------------- structs
class rsrr_c128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class rsrr_fn(C.Structure):
    _fields_ = [("kind", C.c_int32), ("power", C.c_int32), ("param", C.c_double),
                ("scale", rsrr_c128), ("shift", rsrr_c128)]


# void (*)(int32_t term, const rsrr_c128 *z, int64_t count, rsrr_c128 *out, void *user)
rsrr_fn_callback = C.CFUNCTYPE(None, C.c_int32, C.POINTER(rsrr_c128), C.c_int64,
                               C.POINTER(rsrr_c128), C.c_void_p)


class rsrr_nep(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int32), ("kind", C.c_int32),
                ("row_ptr", C.POINTER(C.c_int64)), ("col_idx", C.POINTER(C.c_int32)),
                ("values", C.POINTER(C.c_double)), ("fn", rsrr_fn * RSRR_MAX_TERMS),
                ("points", C.POINTER(C.c_double)), ("diag", C.c_double),
                ("values_complex", C.c_int32), ("reserved", C.c_int32),
                ("dense", C.POINTER(C.POINTER(rsrr_c128))), ("callback", rsrr_fn_callback),
                ("callback_user", C.c_void_p)]


class rsrr_region(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nx", C.c_int32), ("center", rsrr_c128),
                ("a", C.c_double), ("b", C.c_double), ("points", C.POINTER(rsrr_c128))]


class rsrr_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_refine", C.c_int32), ("eta_tol", C.c_double),
                ("delta", C.c_double), ("delta_floor", C.c_double), ("tol_gap", C.c_double),
                ("res_tol", C.c_double), ("NQ", C.c_int32), ("KQ", C.c_int32),
                ("host_threads", C.c_int32), ("timing", C.c_int32), ("gemm", C.c_int32),
                ("flags", C.c_int32), ("seed", C.c_uint64), ("mem_budget_bytes", C.c_int64),
                ("method", C.c_int32), ("K", C.c_int32), ("refine", C.c_int32), ("gmres_m", C.c_int32),
                ("chunk_points", C.c_int32), ("reserved", C.c_int32)]


class rsrr_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("N", C.c_int32), ("L", C.c_int32), ("m", C.c_int32),
                ("kl", C.c_int32), ("ku", C.c_int32), ("refine_sweeps", C.c_int32),
                ("converged", C.c_int32), ("singular_point", C.c_int32), ("k", C.c_int32),
                ("kc", C.c_int32), ("max_eta", C.c_double), ("sigma1", C.c_double),
                ("sigmak", C.c_double), ("device_bytes", C.c_size_t),
                ("launches", C.c_int64), ("stage_ms", C.c_double * 6),
                ("gemm_flops", C.c_double), ("gemm_ms", C.c_double),
                ("tc_flops", C.c_double), ("tc_ms", C.c_double)]


class rsrr_result(C.Structure):
    _fields_ = [("count", C.c_int32), ("nbar", C.c_int32), ("gmax", C.c_double),
                ("lam", C.POINTER(rsrr_c128)), ("res", C.POINTER(C.c_double)),
                ("V", C.POINTER(rsrr_c128))]


class rsrr_server_opts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("keep", C.c_int32), ("mem_budget_bytes", C.c_int64),
                ("device", C.c_int32), ("reserved", C.c_int32)]


class rsrr_reply(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("count", C.c_int32),
                ("nbar", C.c_int32), ("k", C.c_int32), ("refine_sweeps", C.c_int32),
                ("gmax", C.c_double), ("max_eta", C.c_double), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("t_sample", C.c_double),
                ("t_project", C.c_double), ("t_solve", C.c_double), ("device_bytes", C.c_size_t),
                ("n", C.c_int64), ("lam", C.POINTER(rsrr_c128)), ("res", C.POINTER(C.c_double)),
                ("V", C.POINTER(rsrr_c128)), ("error", C.c_char_p)]


class rsrr_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("queued", C.c_int32), ("active", C.c_int32), ("peak_active", C.c_int32),
                ("reserved", C.c_int32), ("used_bytes", C.c_size_t), ("peak_bytes", C.c_size_t),
                ("budget_bytes", C.c_size_t), ("now", C.c_double)]


_h = C.c_void_p
_p = C.c_void_p


def _sig(name, restype, argtypes):
    f = getattr(_lib, name)
    f.restype = restype
    f.argtypes = argtypes
    return f


rsrr_opts_default = _sig("rsrr_opts_default", None, [C.POINTER(rsrr_opts)])
rsrr_create = _sig("rsrr_create", C.c_int, [C.POINTER(rsrr_nep), C.POINTER(rsrr_region),
                                            C.c_int32, C.c_int32, C.POINTER(rsrr_opts),
                                            C.POINTER(_h)])
rsrr_set_probe = _sig("rsrr_set_probe", C.c_int, [_h, _p, C.c_int32, _p])
rsrr_sample = _sig("rsrr_sample", C.c_int, [_h, _p])
rsrr_check = _sig("rsrr_check", C.c_int, [_h, _p])
rsrr_add_points = _sig("rsrr_add_points", C.c_int, [_h, _p, C.c_int32, _p])
rsrr_sample_batch = _sig("rsrr_sample_batch", C.c_int, [C.POINTER(_h), C.c_int32, _p])


def sample_batch(solvers, stream=None):
    """rsrr_sample_batch over several Solver objects (band path)."""
    arr = (_h * len(solvers))(*[sv.h for sv in solvers])
    st = rsrr_sample_batch(arr, len(solvers), _stream_handle(stream))
    if st != RSRR_OK:
        raise RSRRError(st, rsrr_last_error(None).decode())
    return st
rsrr_project = _sig("rsrr_project", C.c_int, [_h, _p])
rsrr_solve = _sig("rsrr_solve", C.c_int, [_h, C.POINTER(rsrr_result)])
rsrr_get_samples = _sig("rsrr_get_samples", C.c_int, [_h, _p, C.c_int32, _p])
rsrr_get_eta = _sig("rsrr_get_eta", C.c_int, [_h, _p])
rsrr_get_Q = _sig("rsrr_get_Q", C.c_int, [_h, _p, C.c_int32, _p])
rsrr_get_projected = _sig("rsrr_get_projected", C.c_int, [_h, _p, C.c_int32, _p])
rsrr_get_points = _sig("rsrr_get_points", C.c_int, [_h, _p])
rsrr_copy_result = _sig("rsrr_copy_result", C.c_int,
                        [_h, C.c_int32, C.POINTER(C.c_int32), _p, _p, _p])
rsrr_get_stats = _sig("rsrr_get_stats", C.c_int, [_h, C.POINTER(rsrr_stats)])
rsrr_last_error = _sig("rsrr_last_error", C.c_char_p, [_h])
rsrr_destroy = _sig("rsrr_destroy", None, [_h])
rsrr_solve_band_noalloc = _sig("rsrr_solve_band_noalloc", C.c_int,
                               [C.c_int64, C.c_int32, C.c_int32, _p, C.c_int32, _p, _p, _p])
rsrr_estimate_bytes = _sig("rsrr_estimate_bytes", C.c_int,
                           [C.POINTER(rsrr_nep), C.POINTER(rsrr_region), C.c_int32, C.c_int32,
                            C.POINTER(rsrr_opts), C.POINTER(C.c_size_t)])
rsrr_server_opts_default = _sig("rsrr_server_opts_default", None, [C.POINTER(rsrr_server_opts)])
rsrr_server_create = _sig("rsrr_server_create", C.c_int, [C.POINTER(rsrr_server_opts), C.POINTER(_h)])
rsrr_server_submit = _sig("rsrr_server_submit", C.c_int,
                          [_h, C.POINTER(rsrr_nep), C.POINTER(rsrr_region), C.c_int32, C.c_int32,
                           C.POINTER(rsrr_opts), _p, C.POINTER(C.c_int64)])
rsrr_server_wait = _sig("rsrr_server_wait", C.c_int, [_h, C.c_int64, C.c_double, C.POINTER(rsrr_reply)])
rsrr_server_handle = _sig("rsrr_server_handle", _h, [_h, C.c_int64])
rsrr_server_release = _sig("rsrr_server_release", C.c_int, [_h, C.c_int64])
rsrr_server_get_stats = _sig("rsrr_server_get_stats", C.c_int, [_h, C.POINTER(rsrr_server_stats)])
rsrr_server_destroy = _sig("rsrr_server_destroy", None, [_h])
rsrr_zgemm = _sig("rsrr_zgemm", C.c_int,
                  [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _p, C.c_int64, _p, C.c_int64, _p,
                   C.c_int64, C.c_double, C.c_double, C.c_int32, C.c_int32, C.c_size_t, _p])
rsrr_check_wait_timeout = _sig("rsrr_check_wait_timeout", C.c_int, [C.c_int32, _p])
rsrr_describe = _sig("rsrr_describe", C.c_int,
                     [C.POINTER(rsrr_nep), C.POINTER(rsrr_region), C.c_int32, C.c_int32,
                      C.POINTER(rsrr_opts), _p, _p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)])


class RSRRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(buf):
    """Device pointer of a torch tensor, or address of a numpy array."""
    if hasattr(buf, "data_ptr"):
        return C.c_void_p(buf.data_ptr())
    return buf.ctypes.data_as(C.c_void_p)


def default_opts(**kw) -> rsrr_opts:
    o = rsrr_opts()
    rsrr_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _fn_struct(fn):
    sc = complex(fn.scale)
    sh = complex(getattr(fn, "shift", 0.0))
    return rsrr_fn(int(fn.kind), int(getattr(fn, "power", 0)), float(fn.param),
                   rsrr_c128(sc.real, sc.imag), rsrr_c128(sh.real, sh.imag))


def _make_callback(fns, keep):
    """One C callback for the problem's RSRR_F_CALLBACK terms: term i is
    evaluated by fns[i].callback(z) (a numpy vector of points)."""
    def cb(term, zp, count, outp, user):
        z = np.ctypeslib.as_array(C.cast(zp, C.POINTER(C.c_double)), shape=(count * 2,)).view(np.complex128)
        out = np.ctypeslib.as_array(C.cast(outp, C.POINTER(C.c_double)), shape=(count * 2,)).view(np.complex128)
        out[:] = np.asarray(fns[term].callback(z.copy()), dtype=np.complex128)
    f = rsrr_fn_callback(cb)
    keep.append(f)
    return f


def describe(prob):
    """rsrr_nep and rsrr_region structures for a problem description (see
    Solver), plus the objects they point into (keep them alive while the
    structures, or a handle built from them, are in use)."""
    keep = []
    nep = rsrr_nep()
    nep.n = int(prob.n)
    fns = getattr(prob, "fns", [])
    if getattr(prob, "As", None) is not None:
        nep.kind = RSRR_NEP_DENSE
        nep.m = len(prob.As)
        mats = [np.asfortranarray(np.asarray(A, dtype=np.complex128)) for A in prob.As]
        keep += mats
        ptrs = (C.POINTER(rsrr_c128) * len(mats))(*[m.ctypes.data_as(C.POINTER(rsrr_c128)) for m in mats])
        keep.append(ptrs)
        nep.dense = C.cast(ptrs, C.POINTER(C.POINTER(rsrr_c128)))
    elif getattr(prob, "points", None) is not None and not hasattr(prob, "row_ptr"):
        pts = np.ascontiguousarray(np.asarray(prob.points, dtype=np.float64))
        keep.append(pts)
        nep.kind = RSRR_NEP_HELMHOLTZ
        nep.points = pts.ctypes.data_as(C.POINTER(C.c_double))
        nep.diag = float(prob.diag)
        fns = []
    else:
        row_ptr = np.ascontiguousarray(prob.row_ptr, dtype=np.int64)
        col_idx = np.ascontiguousarray(prob.col_idx, dtype=np.int32)
        cplx = any(np.iscomplexobj(v) for v in prob.values)
        dt = np.complex128 if cplx else np.float64
        values = np.ascontiguousarray(np.concatenate([np.asarray(v, dtype=dt) for v in prob.values]))
        keep += [row_ptr, col_idx, values]
        nep.kind = RSRR_NEP_SPARSE
        nep.m = len(prob.values)
        nep.values_complex = 1 if cplx else 0
        nep.row_ptr = row_ptr.ctypes.data_as(C.POINTER(C.c_int64))
        nep.col_idx = col_idx.ctypes.data_as(C.POINTER(C.c_int32))
        nep.values = values.ctypes.data_as(C.POINTER(C.c_double))
    for i, fn in enumerate(fns):
        nep.fn[i] = _fn_struct(fn)
    if any(int(fn.kind) == RSRR_F_CALLBACK for fn in fns):
        nep.callback = _make_callback(fns, keep)
    reg = rsrr_region()
    r = prob.region
    reg.center = rsrr_c128(complex(r.center).real, complex(r.center).imag)
    reg.a, reg.b = float(r.a), float(r.b)
    if getattr(r, "kind", "ellipse") == "points":
        reg.kind = RSRR_REGION_POINTS
        pz = np.ascontiguousarray(np.asarray(r.points, dtype=np.complex128))
        keep.append(pz)
        reg.points = pz.ctypes.data_as(C.POINTER(rsrr_c128))
    elif getattr(r, "kind", "ellipse") == "interval":
        reg.kind = RSRR_REGION_INTERVAL
    elif getattr(r, "kind", "ellipse") == "rect":
        reg.kind = RSRR_REGION_RECT
        reg.nx = int(r.nx)
        if getattr(r, "points", None) is not None:
            pz = np.ascontiguousarray(np.asarray(r.points, dtype=np.complex128))
            keep.append(pz)
            reg.points = pz.ctypes.data_as(C.POINTER(rsrr_c128))
    else:
        reg.kind = RSRR_REGION_ELLIPSE
    return nep, reg, keep


def estimate_bytes(prob, opts: rsrr_opts | None = None, N=None, L=None) -> int:
    """Device bytes a handle for `prob` would hold (no GPU needed)."""
    nep, reg, keep = describe(prob)
    o = opts if opts is not None else default_opts()
    b = C.c_size_t(0)
    st = rsrr_estimate_bytes(C.byref(nep), C.byref(reg), int(N if N is not None else prob.N),
                             int(L if L is not None else prob.L), C.byref(o), C.byref(b))
    if st != RSRR_OK:
        raise RSRRError(st, rsrr_last_error(None).decode())
    return int(b.value)


def prepared(prob, opts: rsrr_opts | None = None, N=None, L=None):
    """What rsrr_create prepares on the host for `prob` (no GPU needed):
    sampling points z (N), coefficient table (N x m; None for the dense
    kind) and the detected half-bandwidths (kl, ku)."""
    nep, reg, keep = describe(prob)
    o = opts if opts is not None else default_opts()
    N = int(N if N is not None else prob.N)
    L = int(L if L is not None else prob.L)
    dense = nep.kind == RSRR_NEP_HELMHOLTZ
    z = np.zeros(N, dtype=np.complex128)
    # held terms: a term with complex sparse values may be held as two
    mh = 2 * nep.m if nep.values_complex else nep.m
    coef = None if dense else np.zeros((N, mh), dtype=np.complex128)
    kl, ku = C.c_int32(-1), C.c_int32(-1)
    st = rsrr_describe(C.byref(nep), C.byref(reg), N, L, C.byref(o), z.ctypes.data,
                       None if coef is None else coef.ctypes.data, C.byref(kl), C.byref(ku))
    if st != RSRR_OK:
        raise RSRRError(st, rsrr_last_error(None).decode())
    if coef is not None and nep.values_complex:
        # keep the held terms' columns (terms whose imaginary parts are all
        # zero are held once)
        held = []
        for v in prob.values:
            held.append(True)
            held.append(bool(np.any(np.asarray(v).imag != 0)))
        cols = [c for c, h in enumerate(held) if h]
        flat = coef.reshape(-1)[:N * len(cols)].reshape(N, len(cols))
        coef = flat
    return z, coef, (kl.value, ku.value)


def _complex_array(ptr, count):
    if count == 0:
        return np.zeros(0, dtype=np.complex128)
    return np.ctypeslib.as_array(C.cast(ptr, C.POINTER(C.c_double)), shape=(count * 2,)).copy() \
        .view(np.complex128)


class Server:
    """Request server (rsrr_server_*): submit whole RSRR solves, wait for
    their replies.  Problems are described as for Solver."""

    def __init__(self, slots=4, mem_budget_bytes=None, keep=False, device=-1):
        o = rsrr_server_opts()
        rsrr_server_opts_default(C.byref(o))
        o.slots = int(slots)
        o.keep = 1 if keep else 0
        o.device = int(device)
        if mem_budget_bytes is not None:
            o.mem_budget_bytes = int(mem_budget_bytes)
        h = _h()
        st = rsrr_server_create(C.byref(o), C.byref(h))
        if st != RSRR_OK:
            raise RSRRError(st, rsrr_last_error(None).decode())
        self.h = h

    def submit(self, prob, opts: rsrr_opts | None = None, U=None, N=None, L=None) -> int:
        nep, reg, keep = describe(prob)
        o = opts if opts is not None else default_opts()
        N = int(N if N is not None else prob.N)
        L = int(L if L is not None else prob.L)
        if U is None:
            U = getattr(prob, "U", None)
        up = None
        if U is not None:
            Uf = np.asfortranarray(np.asarray(U, dtype=np.complex128))
            assert Uf.shape == (int(prob.n), L)
            keep.append(Uf)
            up = Uf.ctypes.data_as(C.c_void_p)
        rid = C.c_int64(0)
        st = rsrr_server_submit(self.h, C.byref(nep), C.byref(reg), N, L, C.byref(o), up, C.byref(rid))
        if st != RSRR_OK:
            raise RSRRError(st, rsrr_last_error(None).decode())
        return int(rid.value)

    def wait(self, rid: int, timeout: float = -1.0) -> dict | None:
        """The reply of request `rid` as a dict, or None on timeout."""
        r = rsrr_reply()
        st = rsrr_server_wait(self.h, int(rid), float(timeout), C.byref(r))
        if st == RSRR_ETIMEOUT:
            return None
        if st != RSRR_OK:
            raise RSRRError(st, rsrr_last_error(None).decode())
        cnt, n = r.count, r.n
        lam = _complex_array(r.lam, cnt)
        res = np.ctypeslib.as_array(r.res, shape=(cnt,)).copy() if cnt else np.zeros(0)
        V = _complex_array(r.V, cnt * n).reshape(cnt, n).T if cnt else np.zeros((n, 0), np.complex128)
        return dict(id=r.id, status=r.status, count=cnt, nbar=r.nbar, k=r.k,
                    refine_sweeps=r.refine_sweeps, gmax=r.gmax, max_eta=r.max_eta,
                    t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done,
                    t_sample=r.t_sample, t_project=r.t_project, t_solve=r.t_solve,
                    device_bytes=r.device_bytes, lam=lam, res=res, V=V,
                    error=(r.error or b"").decode())

    def handle(self, rid: int):
        return rsrr_server_handle(self.h, int(rid))

    def release(self, rid: int):
        st = rsrr_server_release(self.h, int(rid))
        if st != RSRR_OK:
            raise RSRRError(st, rsrr_last_error(None).decode())

    def stats(self) -> dict:
        s = rsrr_server_stats()
        st = rsrr_server_get_stats(self.h, C.byref(s))
        if st != RSRR_OK:
            raise RSRRError(st, rsrr_last_error(None).decode())
        return {f: getattr(s, f) for f, _ in rsrr_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            rsrr_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owns one rsrr_t handle built from a problem description: either
    n, row_ptr, col_idx, values (list of m arrays), fns (kind, param, scale)
    for T(z) = sum_i f_i(z) A_i, or n, points (n x 3), diag for the dense
    Helmholtz kernel; plus region (center, a, b, kind, points), N, L."""

    def __init__(self, prob, opts: rsrr_opts | None = None, N: int | None = None,
                 L: int | None = None):
        self.prob = prob
        self.N = int(N if N is not None else prob.N)
        self.L = int(L if L is not None else prob.L)
        self.n = int(prob.n)
        nep, reg, self._keep = describe(prob)
        self.dense = nep.kind in (RSRR_NEP_HELMHOLTZ, RSRR_NEP_DENSE)
        self.opts = opts if opts is not None else default_opts()
        h = _h()
        st = rsrr_create(C.byref(nep), C.byref(reg), self.N, self.L, C.byref(self.opts),
                         C.byref(h))
        if st != RSRR_OK:
            raise RSRRError(st, rsrr_last_error(None).decode())
        self.h = h
        if getattr(prob, "U", None) is not None:
            self.set_probe(prob.U)

    # -------------------------------------------------------------- helpers
    def _check(self, st, ok=(RSRR_OK,)):
        if st not in ok:
            raise RSRRError(st, rsrr_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            rsrr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- calls
    def set_probe(self, U, stream=None):
        if hasattr(U, "data_ptr"):
            return self._check(rsrr_set_probe(self.h, _ptr(U), 1, _stream_handle(stream)))
        Uf = np.asfortranarray(np.asarray(U, dtype=np.complex128))
        assert Uf.shape == (self.n, self.L)
        return self._check(rsrr_set_probe(self.h, Uf.ctypes.data_as(C.c_void_p), 0, None))

    def sample(self, stream=None):
        return self._check(rsrr_sample(self.h, _stream_handle(stream)))

    def add_points(self, z_new, stream=None):
        """Appends sampling points and samples only them (rsrr_add_points)."""
        z = np.ascontiguousarray(np.asarray(z_new, dtype=np.complex128).ravel())
        st = self._check(rsrr_add_points(self.h, z.ctypes.data_as(C.c_void_p), len(z), _stream_handle(stream)))
        self.N += len(z)
        return st

    def check(self, stream=None):
        return self._check(rsrr_check(self.h, _stream_handle(stream)))

    def check_status(self, stream=None):
        return rsrr_check(self.h, _stream_handle(stream))

    def project(self, stream=None):
        return self._check(rsrr_project(self.h, _stream_handle(stream)))

    def samples(self, out=None, stream=None):
        """S (n x N*L) as a numpy array, or into a device tensor `out`."""
        if out is not None:
            self._check(rsrr_get_samples(self.h, _ptr(out), 1, _stream_handle(stream)))
            return out
        S = np.empty((self.N * self.L, self.n), dtype=np.complex128)
        self._check(rsrr_get_samples(self.h, S.ctypes.data_as(C.c_void_p), 0,
                                     _stream_handle(stream)))
        return S.T

    def eta(self):
        e = np.empty(self.N * self.L, dtype=np.float64)
        self._check(rsrr_get_eta(self.h, e.ctypes.data_as(C.c_void_p)))
        return e

    def points(self):
        z = np.empty(self.N, dtype=np.complex128)
        self._check(rsrr_get_points(self.h, z.ctypes.data_as(C.c_void_p)))
        return z

    def stats(self) -> dict:
        s = rsrr_stats()
        self._check(rsrr_get_stats(self.h, C.byref(s)))
        d = {f: getattr(s, f) for f, _ in rsrr_stats._fields_}
        d["stage_ms"] = list(s.stage_ms)
        return d

    def Q(self, out=None, stream=None):
        k = self.stats()["k"]
        if out is not None:
            self._check(rsrr_get_Q(self.h, _ptr(out), 1, _stream_handle(stream)))
            return out
        Q = np.empty((k, self.n), dtype=np.complex128)
        self._check(rsrr_get_Q(self.h, Q.ctypes.data_as(C.c_void_p), 0, _stream_handle(stream)))
        return Q.T

    def projected(self, out=None, stream=None):
        st = self.stats()
        k, m = st["k"], st["m"]
        if out is not None:
            self._check(rsrr_get_projected(self.h, _ptr(out), 1, _stream_handle(stream)))
            return out
        P = np.empty((m, k, k), dtype=np.complex128)
        self._check(rsrr_get_projected(self.h, P.ctypes.data_as(C.c_void_p), 0,
                                       _stream_handle(stream)))
        return [P[i].T.copy() for i in range(m)]

    def copy_result(self):
        """The last rsrr_solve's eigenpairs through rsrr_copy_result (caller buffers)."""
        cnt = C.c_int32(0)
        st = rsrr_copy_result(self.h, 0, C.byref(cnt), None, None, None)
        if st not in (RSRR_OK, RSRR_EINVAL):
            self._check(st)
        k = cnt.value
        lam = np.zeros(k, dtype=np.complex128)
        res = np.zeros(k, dtype=np.float64)
        V = np.zeros((k, self.n), dtype=np.complex128)
        self._check(rsrr_copy_result(self.h, k, C.byref(cnt), lam.ctypes.data_as(C.c_void_p),
                                     res.ctypes.data_as(C.c_void_p), V.ctypes.data_as(C.c_void_p)))
        return dict(lam=lam, res=res, V=V.T)

    def solve(self) -> dict:
        r = rsrr_result()
        st = self._check(rsrr_solve(self.h, C.byref(r)), ok=(RSRR_OK, RSRR_WGAP))
        cnt = r.count
        lam = np.ctypeslib.as_array(C.cast(r.lam, C.POINTER(C.c_double)), shape=(cnt * 2,)).copy() \
            if cnt else np.zeros(0)
        lam = lam.view(np.complex128) if cnt else np.zeros(0, dtype=np.complex128)
        res = np.ctypeslib.as_array(r.res, shape=(cnt,)).copy() if cnt else np.zeros(0)
        if cnt:
            V = np.ctypeslib.as_array(C.cast(r.V, C.POINTER(C.c_double)),
                                      shape=(cnt * self.n * 2,)).copy().view(np.complex128)
            V = V.reshape(cnt, self.n).T
        else:
            V = np.zeros((self.n, 0), dtype=np.complex128)
        return dict(status=st, lam=lam, res=res, V=V, nbar=r.nbar, gmax=r.gmax)
