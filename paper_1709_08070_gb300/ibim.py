"""Thin ctypes binding of the C ABI in ``include/ibim.h`` (argument marshalling only).

Every compute step runs in ``libibim.so`` (hand-written sm_103a CUDA).  There
is no CPU fallback: importing this module raises when the library has not been
built, and the entry points raise ``IbimError`` on any non-OK status.
Device buffers are passed as torch CUDA tensors (float64, contiguous) or raw
integer device pointers; the stream is the current torch stream unless given.
"""
import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "IbimError", "Phys", "SolveOpts", "SolveInfo", "lib", "library_path",
    "ibim_build", "ibim_get_levelset", "ibim_build_sphere", "ibim_build_from_nodes", "ibim_set_charges", "ibim_num_nodes", "ibim_get_nodes",
    "ibim_matvec", "ibim_matvec_host", "ibim_rhs", "ibim_energy", "ibim_area", "ibim_solve", "ibim_solve_host", "ibim_solve_batch",
    "ibim_timing_enable", "ibim_timing_reset", "ibim_timing_get", "ibim_destroy", "ibim_last_error",
    "ibim_matvec_noalloc", "IBIM_NOALLOC_MAX_NODES", "ibim_autotune", "ibim_set_f32_variant", "ibim_f32_variants",
    "IBIM_F64", "IBIM_F32C", "Context", "KCAL_PER_E2_A", "WarmStartNet", "IBIM_WS_NPARAMS",
    "ibim_get_curvature", "ibim_set_jacobian", "ibim_get_jacobian", "ibim_solve_extrapolated",
    "IBIM_F32T", "IBIM_FF", "ibim_treecode_setup", "ibim_treecode_info", "ibim_treecode_plan",
]

IBIM_F64 = 64
IBIM_FF = 65
IBIM_F32C = 32
IBIM_F32T = 33
IBIM_NOALLOC_MAX_NODES = 131072
IBIM_WS_NPARAMS = 4930
IBIM_WS_NFEATURES = 9
KCAL_PER_E2_A = 4.0 * np.pi * 332.0637

_STATUS = {0: "IBIM_OK", 1: "IBIM_ERR_ARG", 2: "IBIM_ERR_EMPTY_BAND", 3: "IBIM_ERR_NONFINITE",
           4: "IBIM_ERR_CUDA", 5: "IBIM_ERR_NOT_CONVERGED", 6: "IBIM_ERR_DEVICE_TIMEOUT", 7: "IBIM_ERR_STATE"}


class IbimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class Phys(ctypes.Structure):
    _fields_ = [("eps_in", ctypes.c_double), ("eps_out", ctypes.c_double), ("kappa", ctypes.c_double),
                ("tau", ctypes.c_double), ("tube_rule", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("restart", ctypes.c_int), ("start", ctypes.c_int), ("certify", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("converged", ctypes.c_int),
                ("relres", ctypes.c_double), ("gpol", ctypes.c_double), ("gpol_kcal", ctypes.c_double),
                ("area", ctypes.c_double), ("matvecs_f32", ctypes.c_int64), ("matvecs_f64", ctypes.c_int64)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


_V = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)
_IP = ctypes.POINTER(ctypes.c_int)
_CTXP = ctypes.POINTER(_V)
_SIGS = {
    "ibim_build_sphere": [ctypes.c_double, _D, _D, ctypes.c_double, ctypes.c_double, _V, _CTXP],
    "ibim_build_from_nodes": [ctypes.c_int64, _D, _D, _D, ctypes.c_double, _V, _CTXP],
    "ibim_set_charges": [_V, ctypes.c_int64, _D, _D],
    "ibim_num_nodes": [_V, _I64P],
    "ibim_get_nodes": [_V, _D, _D, _D, _D, ctypes.POINTER(ctypes.c_int32)],
    "ibim_matvec": [_V, ctypes.POINTER(Phys), ctypes.c_int, _V, _V],
    "ibim_matvec_host": [_V, ctypes.POINTER(Phys), ctypes.c_int, _D, _D],
    "ibim_rhs": [_V, ctypes.c_double, _V],
    "ibim_energy": [_V, ctypes.POINTER(Phys), ctypes.c_int, _V, _V, _D],
    "ibim_area": [_V, _D],
    "ibim_solve": [_V, ctypes.POINTER(Phys), ctypes.POINTER(SolveOpts), _V, ctypes.POINTER(SolveInfo)],
    "ibim_solve_host": [_V, ctypes.POINTER(Phys), ctypes.POINTER(SolveOpts), ctypes.c_int64, _D, _D, _D,
                        ctypes.POINTER(SolveInfo)],
    "ibim_timing_enable": [_V, ctypes.c_int],
    "ibim_timing_reset": [_V],
    "ibim_timing_get": [_V, _D, _I64P, _I64P, _I64P],
    "ibim_matvec_noalloc": [ctypes.c_int64, _V, _V, _V, ctypes.POINTER(Phys), _V, _V, _V],
    "ibim_autotune": [_V, ctypes.POINTER(Phys), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _D],
    "ibim_set_f32_variant": [_V, ctypes.c_int, ctypes.c_int],
    "ibim_treecode_setup": [_V, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int],
    "ibim_treecode_info": [_V, _I64P, _I64P, _I64P, _I64P, _I64P],
    "ibim_treecode_plan": [_D, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int, _I64P, _I64P,
                           ctypes.POINTER(ctypes.c_int32), _I64P, ctypes.POINTER(ctypes.c_int32)],
    "ibim_f32_variant_info": [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "ibim_build": [_D, _D, _D, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double, _V, _CTXP],
    "ibim_get_levelset": [_V, _I64P, _I64P, _D],
    "ibim_solve_batch": [ctypes.c_int, ctypes.POINTER(_V), ctypes.POINTER(Phys), ctypes.POINTER(SolveOpts),
                         ctypes.POINTER(_V), ctypes.POINTER(SolveInfo)],
    "ibim_get_curvature": [_V, _D],
    "ibim_set_jacobian": [_V, ctypes.c_int],
    "ibim_solve_extrapolated": [_V, ctypes.POINTER(Phys), ctypes.POINTER(SolveOpts), _V, ctypes.POINTER(SolveInfo)],
    "ibim_get_jacobian": [_V, _D],
    "ibim_wsnet_create": [ctypes.c_uint64, _V, _CTXP],
    "ibim_wsnet_get_params": [_V, ctypes.POINTER(ctypes.c_float)],
    "ibim_wsnet_set_params": [_V, ctypes.POINTER(ctypes.c_float)],
    "ibim_wsnet_features": [_V, _V, ctypes.POINTER(Phys), ctypes.POINTER(ctypes.c_float), _D],
    "ibim_wsnet_add_example": [_V, _V, ctypes.POINTER(Phys), _V],
    "ibim_wsnet_num_examples": [_V, _I64P],
    "ibim_wsnet_gradient": [_V, ctypes.c_int64, ctypes.c_int64, _D, ctypes.POINTER(ctypes.c_float)],
    "ibim_wsnet_train": [_V, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D],
    "ibim_wsnet_predict": [_V, _V, ctypes.POINTER(Phys), _V],
    "ibim_debug_raise_device_error": [_V, ctypes.c_int],
    "ibim_batch_variant_info": [ctypes.c_int, _IP, _IP, _IP, _IP],
    "ibim_set_batch_variant": [ctypes.c_int],
    "ibim_set_ff_kernel": [_V, ctypes.c_int],
}

_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load libibim.so (raises when it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError("libibim.so is not built (%s); run __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.ibim_last_error.restype = ctypes.c_char_p
        L.ibim_last_error.argtypes = []
        L.ibim_f32_variant_count.restype = ctypes.c_int
        L.ibim_f32_variant_count.argtypes = []
        L.ibim_batch_variant_count.restype = ctypes.c_int
        L.ibim_batch_variant_count.argtypes = []
        L.ibim_wsnet_destroy.restype = None
        L.ibim_wsnet_destroy.argtypes = [_V]
        L.ibim_destroy.restype = None
        L.ibim_destroy.argtypes = [_V]
        _lib = L
    return _lib


def ibim_last_error():
    return lib().ibim_last_error().decode()


def _check(status):
    if status != 0:
        raise IbimError(status, ibim_last_error())
    return status


def _dptr(x):
    """Device pointer of a torch CUDA tensor (float64, contiguous) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return x.data_ptr()


def _host(a, dtype=np.float64):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _stream(stream):
    if stream is not None:
        return int(stream)
    import torch
    return torch.cuda.current_stream().cuda_stream


def _phys(p):
    if isinstance(p, Phys):
        return p
    if isinstance(p, dict):
        return Phys(p["eps_in"], p["eps_out"], p["kappa"], p["tau"], p.get("tube_rule", 0))
    return Phys(*p)


# ----------------------------------------------------------------- raw calls

def ibim_build(xyz, radii, charges, probe, h, band_eps, stream=None):
    z = _host(xyz).reshape(-1, 3)
    r = _host(radii).reshape(-1)
    q = None if charges is None else _host(charges).reshape(-1)
    ctx = _V()
    _check(lib().ibim_build(z.ctypes.data_as(_D), r.ctypes.data_as(_D), None if q is None else q.ctypes.data_as(_D),
                            r.shape[0], float(probe), float(h), float(band_eps), _stream(stream), ctypes.byref(ctx)))
    return ctx


def ibim_get_levelset(ctx):
    lo = (ctypes.c_int64 * 3)()
    n = (ctypes.c_int64 * 3)()
    _check(lib().ibim_get_levelset(ctx, lo, n, None))
    phi = np.empty(n[0] * n[1] * n[2])
    _check(lib().ibim_get_levelset(ctx, lo, n, phi.ctypes.data_as(_D)))
    return list(lo), list(n), phi.reshape(n[2], n[1], n[0])


def ibim_build_sphere(R, centre, origin, h, band_eps, stream=None):
    c = _host(centre)
    o = None if origin is None else _host(origin)
    ctx = _V()
    _check(lib().ibim_build_sphere(float(R), c.ctypes.data_as(_D), None if o is None else o.ctypes.data_as(_D),
                                   float(h), float(band_eps), _stream(stream), ctypes.byref(ctx)))
    return ctx


def ibim_build_from_nodes(xstar, normal, w, h, stream=None):
    xs = _host(xstar).reshape(-1, 3)
    nr = _host(normal).reshape(-1, 3)
    ww = _host(w).reshape(-1)
    ctx = _V()
    _check(lib().ibim_build_from_nodes(xs.shape[0], xs.ctypes.data_as(_D), nr.ctypes.data_as(_D),
                                       ww.ctypes.data_as(_D), float(h), _stream(stream), ctypes.byref(ctx)))
    return ctx


def ibim_set_charges(ctx, z, q):
    z = _host(z).reshape(-1, 3)
    q = _host(q).reshape(-1)
    _check(lib().ibim_set_charges(ctx, q.shape[0], z.ctypes.data_as(_D), q.ctypes.data_as(_D)))


def ibim_num_nodes(ctx):
    n = ctypes.c_int64(0)
    _check(lib().ibim_num_nodes(ctx, ctypes.byref(n)))
    return n.value


def ibim_get_nodes(ctx):
    N = ibim_num_nodes(ctx)
    xs = np.empty((N, 3))
    nr = np.empty((N, 3))
    w = np.empty(N)
    d = np.empty(N)
    ijk = np.empty((N, 3), dtype=np.int32)
    _check(lib().ibim_get_nodes(ctx, xs.ctypes.data_as(_D), nr.ctypes.data_as(_D), w.ctypes.data_as(_D),
                                d.ctypes.data_as(_D), ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return {"xs": xs, "nrm": nr, "w": w, "d": d, "ijk": ijk}


def ibim_matvec(ctx, phys, precision, d_in, d_out):
    p = _phys(phys)
    _check(lib().ibim_matvec(ctx, ctypes.byref(p), int(precision), _dptr(d_in), _dptr(d_out)))


def ibim_matvec_host(ctx, phys, precision, h_in):
    p = _phys(phys)
    x = _host(h_in)
    y = np.empty_like(x)
    _check(lib().ibim_matvec_host(ctx, ctypes.byref(p), int(precision), x.ctypes.data_as(_D),
                                  y.ctypes.data_as(_D)))
    return y


def ibim_rhs(ctx, eps_in, d_g):
    _check(lib().ibim_rhs(ctx, float(eps_in), _dptr(d_g)))


def ibim_energy(ctx, phys, precision, d_p, d_psi_rxn=None):
    p = _phys(phys)
    g = ctypes.c_double(0.0)
    _check(lib().ibim_energy(ctx, ctypes.byref(p), int(precision), _dptr(d_p), _dptr(d_psi_rxn), ctypes.byref(g)))
    return g.value


def ibim_area(ctx):
    a = ctypes.c_double(0.0)
    _check(lib().ibim_area(ctx, ctypes.byref(a)))
    return a.value


def _opts(precision=IBIM_F32C, tol=1e-6, maxit=500, restart=64, start=0, certify=0):
    return SolveOpts(int(precision), float(tol), int(maxit), int(restart), int(start), int(certify))


def ibim_solve(ctx, phys, d_p, allow_not_converged=False, **opts):
    p = _phys(phys)
    o = _opts(**opts)
    info = SolveInfo()
    st = lib().ibim_solve(ctx, ctypes.byref(p), ctypes.byref(o), _dptr(d_p), ctypes.byref(info))
    if not (allow_not_converged and st == 5):
        _check(st)
    return info.as_dict()


def ibim_solve_extrapolated(ctx, phys, d_p, allow_not_converged=False, **opts):
    """Solves with tau and tau/2 and returns the Richardson combination (see include/ibim.h)."""
    p = _phys(phys)
    o = _opts(**opts)
    info = SolveInfo()
    st = lib().ibim_solve_extrapolated(ctx, ctypes.byref(p), ctypes.byref(o), _dptr(d_p), ctypes.byref(info))
    if not (allow_not_converged and st == 5):
        _check(st)
    return info.as_dict()


def ibim_solve_batch(ctxs, physs, d_ps, allow_not_converged=False, **opts):
    """Batched FP32 solve of several contexts; returns a list of info dicts."""
    n = len(ctxs)
    arr_c = (_V * n)(*[c.handle if isinstance(c, Context) else c for c in ctxs])
    arr_p = (Phys * n)(*[_phys(p) for p in physs])
    arr_d = (_V * n)(*[_dptr(d) for d in d_ps])
    infos = (SolveInfo * n)()
    o = _opts(**opts)
    st = lib().ibim_solve_batch(n, arr_c, arr_p, ctypes.byref(o), arr_d, infos)
    if not (allow_not_converged and st == 5):
        _check(st)
    return [infos[i].as_dict() for i in range(n)]


def ibim_solve_host(ctx, phys, z, q, h_p=None, allow_not_converged=False, **opts):
    p = _phys(phys)
    o = _opts(**opts)
    z = _host(z).reshape(-1, 3)
    q = _host(q).reshape(-1)
    info = SolveInfo()
    out = h_p if h_p is not None else np.empty(2 * ibim_num_nodes(ctx))
    st = lib().ibim_solve_host(ctx, ctypes.byref(p), ctypes.byref(o), q.shape[0], z.ctypes.data_as(_D),
                               q.ctypes.data_as(_D), out.ctypes.data_as(_D), ctypes.byref(info))
    if not (allow_not_converged and st == 5):
        _check(st)
    return out, info.as_dict()


def ibim_timing_enable(ctx, enable=True):
    _check(lib().ibim_timing_enable(ctx, 1 if enable else 0))


def ibim_timing_reset(ctx):
    _check(lib().ibim_timing_reset(ctx))


def ibim_timing_get(ctx):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    inter = ctypes.c_int64(0)
    tot = ctypes.c_int64(0)
    _check(lib().ibim_timing_get(ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(inter), ctypes.byref(tot)))
    return {"pair_ms": ms.value, "pair_launches": n.value, "pair_interactions": inter.value,
            "total_launches": tot.value}


def ibim_debug_raise_device_error(ctx, status=6):
    """Sets the device-timeout bit of the context's error word (failure-path test hook)."""
    _check(lib().ibim_debug_raise_device_error(ctx, int(status)))


def ibim_matvec_noalloc(N, d_xstar, d_normal, d_w, phys, d_in, d_out, stream=None):
    """Allocation-free FP32 compensated product from caller-owned device arrays
    (see include/ibim.h); synchronises the stream before returning."""
    p = _phys(phys)
    _check(lib().ibim_matvec_noalloc(int(N), _dptr(d_xstar), _dptr(d_normal), _dptr(d_w), ctypes.byref(p),
                                     _dptr(d_in), _dptr(d_out), _stream(stream)))


def ibim_f32_variants():
    """[(targets_per_thread, min_ctas_per_sm, threads_per_cta, symmetric)] of the compiled FP32 variants."""
    out = []
    for v in range(lib().ibim_f32_variant_count()):
        t, m, w, y = (ctypes.c_int(0) for _ in range(4))
        _check(lib().ibim_f32_variant_info(v, ctypes.byref(t), ctypes.byref(m), ctypes.byref(w), ctypes.byref(y)))
        out.append((t.value, m.value, w.value, y.value))
    return out


def ibim_batch_variants():
    """([(targets_per_thread, threads_per_cta, symmetric)] of the batched pair-kernel variants,
    variant run by the last batched solve of this thread or -1)."""
    out, last = [], ctypes.c_int(-1)
    for v in range(lib().ibim_batch_variant_count()):
        t, w, y = (ctypes.c_int(0) for _ in range(3))
        _check(lib().ibim_batch_variant_info(v, ctypes.byref(t), ctypes.byref(w), ctypes.byref(y), ctypes.byref(last)))
        out.append((t.value, w.value, y.value))
    return out, last.value


def ibim_set_batch_variant(v):
    """Force batched variant v for later batched solves (-1: the measured choice)."""
    _check(lib().ibim_set_batch_variant(int(v)))


def ibim_autotune(ctx, phys):
    """Pick the fastest FP32 pair-kernel variant; returns (variant, ctas_per_sm, ms)."""
    p = _phys(phys)
    t = ctypes.c_int(0)
    b = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(lib().ibim_autotune(ctx, ctypes.byref(p), ctypes.byref(t), ctypes.byref(b), ctypes.byref(ms)))
    return t.value, b.value, ms.value


def ibim_treecode_setup(ctx, theta, tau_max, target_interp=0, order=6):
    """Build the treecode tree and interaction lists (IBIM_F32T operator)."""
    _check(lib().ibim_treecode_setup(ctx, float(theta), float(tau_max), int(order), int(target_interp)))


def ibim_treecode_info(ctx):
    """{'near_steps', 'far_steps', 'interp_steps', 'clusters', 'target_tiles'} of the current treecode setup."""
    v = [ctypes.c_int64(0) for _ in range(5)]
    _check(lib().ibim_treecode_info(ctx, *[ctypes.byref(x) for x in v]))
    return dict(zip(("near_steps", "far_steps", "interp_steps", "clusters", "target_tiles"), (x.value for x in v)))


def ibim_treecode_plan(xyz, theta, tau_max, target_interp=0):
    """Host-only tree and lists of the treecode for nodes xyz (N x 3):
    dict(n_t, clusters, n_real, row_ptr, steps, irow, isrc) (numpy arrays)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    N = xyz.shape[0]
    sizes = np.zeros(5, dtype=np.int64)
    I64 = ctypes.POINTER(ctypes.c_int64)
    I32 = ctypes.POINTER(ctypes.c_int32)
    args = (xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), N, float(theta), float(tau_max), int(target_interp))
    _check(lib().ibim_treecode_plan(*args, sizes.ctypes.data_as(I64), None, None, None, None))
    n_t, ncl, S, I, n_real = (int(v) for v in sizes)
    row_ptr = np.zeros(n_t + 1, dtype=np.int64)
    irow = np.zeros(n_t + 1, dtype=np.int64)
    steps = np.zeros(max(S, 1), dtype=np.int32)
    isrc = np.zeros(max(I, 1), dtype=np.int32)
    _check(lib().ibim_treecode_plan(*args, sizes.ctypes.data_as(I64), row_ptr.ctypes.data_as(I64),
                                    steps.ctypes.data_as(I32), irow.ctypes.data_as(I64), isrc.ctypes.data_as(I32)))
    return dict(n_t=n_t, clusters=ncl, n_real=n_real, row_ptr=row_ptr, steps=steps[:S], irow=irow, isrc=isrc[:I])


def ibim_set_f32_variant(ctx, variant, ctas_per_sm=0):
    _check(lib().ibim_set_f32_variant(ctx, int(variant), int(ctas_per_sm)))


def ibim_set_jacobian(ctx, mode):
    _check(lib().ibim_set_jacobian(ctx, int(mode)))


def ibim_get_jacobian(ctx):
    N = ibim_num_nodes(ctx)
    out = np.empty(N)
    _check(lib().ibim_get_jacobian(ctx, out.ctypes.data_as(_D)))
    return out


def ibim_get_curvature(ctx):
    out = np.empty(ibim_num_nodes(ctx))
    _check(lib().ibim_get_curvature(ctx, out.ctypes.data_as(_D)))
    return out


def _h(c):
    return c.handle if isinstance(c, Context) else c


class WarmStartNet:
    """Owning wrapper of an ibim_wsnet (learned GMRES start, see include/ibim.h)."""

    def __init__(self, seed=0, stream=None):
        h = _V()
        _check(lib().ibim_wsnet_create(int(seed), _stream(stream), ctypes.byref(h)))
        self.handle = h

    def params(self):
        out = np.empty(IBIM_WS_NPARAMS, dtype=np.float32)
        _check(lib().ibim_wsnet_get_params(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def set_params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == IBIM_WS_NPARAMS
        _check(lib().ibim_wsnet_set_params(self.handle, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def features(self, ctx, phys):
        N = ibim_num_nodes(_h(ctx))
        f = np.empty((N, IBIM_WS_NFEATURES), dtype=np.float32)
        sc = np.empty(3)
        p = _phys(phys)
        _check(lib().ibim_wsnet_features(self.handle, _h(ctx), ctypes.byref(p),
                                         f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), sc.ctypes.data_as(_D)))
        return f, sc

    def add_example(self, ctx, phys, d_p):
        p = _phys(phys)
        _check(lib().ibim_wsnet_add_example(self.handle, _h(ctx), ctypes.byref(p), _dptr(d_p)))

    def num_examples(self):
        n = ctypes.c_int64(0)
        _check(lib().ibim_wsnet_num_examples(self.handle, ctypes.byref(n)))
        return n.value

    def gradient(self, first, count):
        g = np.empty(IBIM_WS_NPARAMS, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(lib().ibim_wsnet_gradient(self.handle, int(first), int(count), ctypes.byref(loss),
                                         g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return loss.value, g

    def train(self, steps, batch_nodes=8192, lr=1e-3):
        loss = ctypes.c_double(0.0)
        _check(lib().ibim_wsnet_train(self.handle, int(steps), int(batch_nodes), float(lr), ctypes.byref(loss)))
        return loss.value

    def predict(self, ctx, phys, d_p0):
        p = _phys(phys)
        _check(lib().ibim_wsnet_predict(self.handle, _h(ctx), ctypes.byref(p), _dptr(d_p0)))

    def close(self):
        if self.handle:
            lib().ibim_wsnet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ibim_destroy(ctx):
    if ctx:
        lib().ibim_destroy(ctx)


class Context:
    """Owning wrapper of an ibim_ctx handle (destroyed on close / garbage collection)."""

    def __init__(self, handle):
        self.handle = handle

    @classmethod
    def sphere(cls, R, centre=(0.0, 0.0, 0.0), h=0.25, band_eps=None, origin=None, stream=None):
        return cls(ibim_build_sphere(R, centre, origin, h, 2 * h if band_eps is None else band_eps, stream))

    @classmethod
    def molecule(cls, xyz, radii, charges=None, probe=1.4, h=0.5, band_eps=None, stream=None):
        return cls(ibim_build(xyz, radii, charges, probe, h, 2 * h if band_eps is None else band_eps, stream))

    def levelset(self):
        return ibim_get_levelset(self.handle)

    @classmethod
    def from_nodes(cls, xstar, normal, w, h, stream=None):
        return cls(ibim_build_from_nodes(xstar, normal, w, h, stream))

    @property
    def N(self):
        return ibim_num_nodes(self.handle)

    def nodes(self):
        return ibim_get_nodes(self.handle)

    def set_charges(self, z, q):
        ibim_set_charges(self.handle, z, q)

    def matvec(self, phys, d_in, d_out, precision=IBIM_F32C):
        ibim_matvec(self.handle, phys, precision, d_in, d_out)

    def matvec_host(self, phys, h_in, precision=IBIM_F32C):
        return ibim_matvec_host(self.handle, phys, precision, h_in)

    def rhs(self, eps_in, d_g):
        ibim_rhs(self.handle, eps_in, d_g)

    def energy(self, phys, d_p, d_psi=None, precision=IBIM_F64):
        return ibim_energy(self.handle, phys, precision, d_p, d_psi)

    def area(self):
        return ibim_area(self.handle)

    def solve(self, phys, d_p, **opts):
        return ibim_solve(self.handle, phys, d_p, **opts)

    def solve_extrapolated(self, phys, d_p, **opts):
        return ibim_solve_extrapolated(self.handle, phys, d_p, **opts)

    def solve_host(self, phys, z, q, h_p=None, **opts):
        return ibim_solve_host(self.handle, phys, z, q, h_p, **opts)

    def autotune(self, phys):
        return ibim_autotune(self.handle, phys)

    def curvature(self):
        return ibim_get_curvature(self.handle)

    def set_jacobian(self, mode):
        ibim_set_jacobian(self.handle, mode)

    def jacobian(self):
        return ibim_get_jacobian(self.handle)

    def set_f32_variant(self, variant, ctas_per_sm=0):
        ibim_set_f32_variant(self.handle, variant, ctas_per_sm)

    def set_ff_kernel(self, symmetric):
        """IBIM_FF kernel: 1 symmetric (default), 0 one-directional."""
        _check(lib().ibim_set_ff_kernel(self.handle, int(symmetric)))

    def treecode_setup(self, theta, tau_max, target_interp=0, order=6):
        ibim_treecode_setup(self.handle, theta, tau_max, target_interp, order)

    def treecode_info(self):
        return ibim_treecode_info(self.handle)

    def timing_enable(self, enable=True):
        ibim_timing_enable(self.handle, enable)

    def timing_reset(self):
        ibim_timing_reset(self.handle)

    def timing(self):
        return ibim_timing_get(self.handle)

    def close(self):
        if self.handle:
            ibim_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
