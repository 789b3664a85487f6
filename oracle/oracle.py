"""ctypes wrappers of the FP64 C oracle (test infrastructure only).

Every function takes and returns numpy float64 arrays; node arrays are
(N, 3) projections x*, (N, 3) unit normals n(x*) and (N,) weights
w = J delta_eps(d) h^3.  Vectors of the discrete system are [psi; psin]
(length 2N).  Citations refer to sections/equations of the paper.
"""
import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "Phys", "lib", "num_threads", "set_num_threads", "delta_eps", "pair_kernels", "matvec", "matvec_rows", "dense",
    "rhs", "psi_rxn", "gpol", "area", "sphere_nodes", "gmres", "KCAL_PER_E2_A",
    "ls_grid", "make_grid", "grid_coords", "ls_ses", "ls_steps", "ls_band", "ses_nodes", "jacobian",
    "jacobian_weights", "solve_energy", "extrapolated_energy",
]

# Coulomb constant in kcal mol^-1 Angstrom e^-2 times 4 pi: energies in the
# paper's convention psi = q/(4 pi eps r) (Sec. 4.2) are converted to kcal/mol
# by this factor (a reading: the paper does not print the conversion).
KCAL_PER_E2_A = 4.0 * np.pi * 332.0637


class _Phys(ctypes.Structure):
    _fields_ = [("eps_in", ctypes.c_double), ("eps_out", ctypes.c_double),
                ("kappa", ctypes.c_double), ("tau", ctypes.c_double),
                ("tube_rule", ctypes.c_int)]


class Phys:
    """Physical and regularisation parameters (Sec. 2.1, Sec. 2.2.1)."""

    def __init__(self, eps_in=1.0, eps_out=80.0, kappa=0.1257, tau=0.25, tube_rule=0):
        self.eps_in, self.eps_out, self.kappa, self.tau, self.tube_rule = (
            float(eps_in), float(eps_out), float(kappa), float(tau), int(tube_rule))

    def c(self):
        return _Phys(self.eps_in, self.eps_out, self.kappa, self.tau, self.tube_rule)


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_P = ctypes.POINTER(_Phys)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_delta_eps.restype = ctypes.c_double
        L.orc_delta_eps.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_pair_kernels.restype = ctypes.c_int
        L.orc_pair_kernels.argtypes = [_D, _D, _D, _D, _P, _D]
        L.orc_matvec.restype = None
        L.orc_matvec.argtypes = [ctypes.c_int64, _D, _D, _D, _P, _D, _D]
        L.orc_matvec_rows.restype = None
        L.orc_matvec_rows.argtypes = [ctypes.c_int64, _D, _D, _D, _P, _D, ctypes.c_int64, _I64, _D]
        L.orc_dense.restype = None
        L.orc_dense.argtypes = [ctypes.c_int64, _D, _D, _D, _P, _D]
        L.orc_rhs.restype = None
        L.orc_rhs.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_int64, _D, _D, ctypes.c_double, _D]
        L.orc_psi_rxn.restype = None
        L.orc_psi_rxn.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int64, _D, _P, _D, _D]
        L.orc_gpol.restype = ctypes.c_double
        L.orc_gpol.argtypes = [ctypes.c_int64, _D, _D]
        L.orc_area.restype = ctypes.c_double
        L.orc_area.argtypes = [ctypes.c_int64, _D]
        L.orc_sphere_nodes.restype = ctypes.c_int64
        L.orc_sphere_nodes.argtypes = [ctypes.c_double, _D, _D, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int64, _D, _D, _D, _D, _I32, _D, _D]
        L.orc_gmres.restype = ctypes.c_int
        L.orc_gmres.argtypes = [ctypes.c_int64, _D, _D, _D, _P, _D, _D, ctypes.c_double,
                                ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_num_threads.argtypes = []
        L.orc_set_num_threads.restype = None
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    """Threads of later oracle calls (OpenMP over independent rows)."""
    lib().orc_set_num_threads(int(n))


def delta_eps(eta, eps):
    """Cosine weight of Sec. 3.2."""
    return lib().orc_delta_eps(float(eta), float(eps))


def pair_kernels(x, nx, y, ny, phys):
    """(K11, K12, K21, K22), in_tube for one pair (Sec. 2.2, Sec. 2.2.1)."""
    K = np.zeros(4)
    P = phys.c()
    t = lib().orc_pair_kernels(_d(_f64(x, 3)), _d(_f64(nx, 3)), _d(_f64(y, 3)), _d(_f64(ny, 3)),
                               ctypes.byref(P), _d(K))
    return K, bool(t)


def _geom(xs, nrm, w):
    xs = _f64(xs, (-1, 3))
    nrm = _f64(nrm, (-1, 3))
    w = _f64(w, -1)
    assert xs.shape[0] == nrm.shape[0] == w.shape[0]
    return xs, nrm, w


def matvec(xs, nrm, w, phys, p):
    """(Lambda + K W) p, Sec. 2.2 discrete system / Sec. 3.3."""
    xs, nrm, w = _geom(xs, nrm, w)
    N = w.shape[0]
    p = _f64(p, 2 * N)
    y = np.empty(2 * N)
    P = phys.c()
    lib().orc_matvec(N, _d(xs), _d(nrm), _d(w), ctypes.byref(P), _d(p), _d(y))
    return y


def matvec_rows(xs, nrm, w, phys, p, rows):
    """Rows `rows` of (Lambda + K W) p; returns (y1[rows], y2[rows])."""
    xs, nrm, w = _geom(xs, nrm, w)
    N = w.shape[0]
    p = _f64(p, 2 * N)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(2 * rows.shape[0])
    P = phys.c()
    lib().orc_matvec_rows(N, _d(xs), _d(nrm), _d(w), ctypes.byref(P), _d(p), rows.shape[0],
                          rows.ctypes.data_as(_I64), _d(out))
    return out[0::2].copy(), out[1::2].copy()


def dense(xs, nrm, w, phys):
    """Dense 2N x 2N matrix Lambda + K W (for brute force on tiny inputs)."""
    xs, nrm, w = _geom(xs, nrm, w)
    N = w.shape[0]
    A = np.empty((2 * N, 2 * N))
    P = phys.c()
    lib().orc_dense(N, _d(xs), _d(nrm), _d(w), ctypes.byref(P), _d(A))
    return A


def rhs(xs, nrm, z, q, eps_in):
    """g = [g1; g2] of Sec. 2.2."""
    xs = _f64(xs, (-1, 3))
    nrm = _f64(nrm, (-1, 3))
    z = _f64(z, (-1, 3))
    q = _f64(q, -1)
    N = xs.shape[0]
    g = np.empty(2 * N)
    lib().orc_rhs(N, _d(xs), _d(nrm), z.shape[0], _d(z), _d(q), float(eps_in), _d(g))
    return g


def psi_rxn(xs, nrm, w, z, phys, p):
    """Reaction potential at each charge centre (Sec. 3.5)."""
    xs, nrm, w = _geom(xs, nrm, w)
    z = _f64(z, (-1, 3))
    N = w.shape[0]
    p = _f64(p, 2 * N)
    out = np.empty(z.shape[0])
    P = phys.c()
    lib().orc_psi_rxn(N, _d(xs), _d(nrm), _d(w), z.shape[0], _d(z), ctypes.byref(P), _d(p), _d(out))
    return out


def gpol(q, psi):
    """G_pol = 1/2 sum q_k psi_rxn(z_k) in e^2/Angstrom (Sec. 3.5)."""
    q = _f64(q, -1)
    psi = _f64(psi, -1)
    return lib().orc_gpol(q.shape[0], _d(q), _d(psi))


def area(w):
    """Surface area, the IBIM sum of f = 1 (Sec. 3.4)."""
    w = _f64(w, -1)
    return lib().orc_area(w.shape[0], _d(w))


def sphere_nodes(R, centre=(0.0, 0.0, 0.0), h=0.25, eps=0.75, origin=(0.0, 0.0, 0.0)):
    """Band nodes of an analytic sphere; dict of xs, nrm, w, d, ijk (lexicographic, x fastest)."""
    c = _f64(centre, 3)
    o = _f64(origin, 3)
    L = lib()
    n = L.orc_sphere_nodes(float(R), _d(c), _d(o), float(h), float(eps), 0, None, None, None, None, None, None,
                           None)
    xs = np.empty((n, 3))
    nrm = np.empty((n, 3))
    w = np.empty(n)
    d = np.empty(n)
    ijk = np.empty((n, 3), dtype=np.int32)
    lap = np.empty(n)
    sig2 = np.empty(n)
    n2 = L.orc_sphere_nodes(float(R), _d(c), _d(o), float(h), float(eps), n, _d(xs), _d(nrm), _d(w),
                            _d(d), ijk.ctypes.data_as(_I32), _d(lap), _d(sig2))
    assert n2 == n
    # curv: Laplacian of d at the grid node (twice the mean curvature of the level sphere through it)
    return {"xs": xs, "nrm": nrm, "w": w, "d": d, "ijk": ijk, "curv": lap, "sig2": sig2}


def gmres(xs, nrm, w, phys, g, x0=None, tol=1e-8, restart=100, maxit=500):
    """Restarted GMRES(m), MGS, FP64 (Sec. 3.3).  Returns (x, iters, true_relres, converged)."""
    xs, nrm, w = _geom(xs, nrm, w)
    N = w.shape[0]
    g = _f64(g, 2 * N)
    x = np.zeros(2 * N) if x0 is None else _f64(x0, 2 * N).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    P = phys.c()
    rc = lib().orc_gmres(N, _d(xs), _d(nrm), _d(w), ctypes.byref(P), _d(g), _d(x), float(tol),
                         int(restart), int(maxit), ctypes.byref(it), ctypes.byref(rr))
    return x, it.value, rr.value, rc == 0


# ------------------------------------------------------------- level set (Sec. 3.1-3.2)

class _Grid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int64 * 3), ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double)]


def _ls_lib():
    L = lib()
    if not getattr(L, "_ls_ready", False):
        G = ctypes.POINTER(_Grid)
        L.orc_ls_grid.restype = None
        L.orc_ls_grid.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double, G]
        L.orc_ls_vdw.restype = None
        L.orc_ls_vdw.argtypes = [G, ctypes.c_int64, _D, _D, ctypes.c_double, _D]
        L.orc_ls_eikonal.restype = ctypes.c_int
        L.orc_ls_eikonal.argtypes = [G, _D, ctypes.c_double]
        L.orc_ls_reinit.restype = ctypes.c_int
        L.orc_ls_reinit.argtypes = [G, _D, ctypes.c_double]
        L.orc_ls_cavity.restype = ctypes.c_int64
        L.orc_ls_cavity.argtypes = [G, _D, ctypes.c_double, ctypes.POINTER(ctypes.c_uint8)]
        L.orc_ls_band.restype = ctypes.c_int64
        L.orc_ls_band.argtypes = [G, _D, ctypes.c_double, ctypes.c_int64, _D, _D, _D, _D, _I32, _D, _D]
        L.orc_ls_ses.restype = ctypes.c_int64
        L.orc_ls_ses.argtypes = [G, ctypes.c_int64, _D, _D, ctypes.c_double, ctypes.c_double, _D]
        L._ls_ready = True
    return L


def ls_grid(z, r, probe, h, eps):
    """Grid box of the level-set construction: dict(lo, n, h)."""
    z = _f64(z, (-1, 3))
    r = _f64(r, -1)
    g = _Grid()
    _ls_lib().orc_ls_grid(r.shape[0], _d(z), _d(r), float(probe), float(h), float(eps), ctypes.byref(g))
    return g


def make_grid(lo, n, h):
    """A level-set grid with node (0,0,0) at integer coordinates lo, n nodes per axis, spacing h."""
    g = _Grid()
    for a in range(3):
        g.lo[a] = int(lo[a])
        g.n[a] = int(n[a])
    g.h = float(h)
    return g


def grid_coords(g):
    """Node coordinates (n2, n1, n0, 3) of a level-set grid."""
    ax = [g.h * (g.lo[a] + np.arange(g.n[a])) for a in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


def ls_ses(z, r, probe=1.4, h=0.5, eps=1.0):
    """Stage 1 (Sec. 3.1): phi_SES on the grid.  Returns (grid, phi (n2, n1, n0), changed)."""
    z = _f64(z, (-1, 3))
    r = _f64(r, -1)
    g = ls_grid(z, r, probe, h, eps)
    phi = np.empty(g.n[0] * g.n[1] * g.n[2])
    ch = _ls_lib().orc_ls_ses(ctypes.byref(g), r.shape[0], _d(z), _d(r), float(probe), float(eps), _d(phi))
    return g, phi.reshape(g.n[2], g.n[1], g.n[0]), ch


def ls_steps(z, r, probe=1.4, h=0.5, eps=1.0):
    """Stage 1 step by step: dict of the grids after F, eikonal flow, cavity removal, reinit."""
    z = _f64(z, (-1, 3))
    r = _f64(r, -1)
    L = _ls_lib()
    g = ls_grid(z, r, probe, h, eps)
    M = g.n[0] * g.n[1] * g.n[2]
    shape = (g.n[2], g.n[1], g.n[0])
    F = np.empty(M)
    L.orc_ls_vdw(ctypes.byref(g), r.shape[0], _d(z), _d(r), 2.0 * probe + eps + 6.0 * h, _d(F))
    phi = F - probe
    sas = phi.copy()
    L.orc_ls_eikonal(ctypes.byref(g), _d(phi), float(probe))
    flowed = phi.copy()
    lab = np.zeros(M, dtype=np.uint8)
    ch = L.orc_ls_cavity(ctypes.byref(g), _d(phi), float(eps), lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    cav = phi.copy()
    L.orc_ls_reinit(ctypes.byref(g), _d(phi), float(eps))
    return {"grid": g, "F": F.reshape(shape), "sas": sas.reshape(shape), "flowed": flowed.reshape(shape),
            "labels": lab.reshape(shape), "cavity": cav.reshape(shape), "phi": phi.reshape(shape), "changed": ch}


def ls_band(g, phi, eps):
    """Band nodes of a level-set grid (Sec. 3.2): dict of xs, nrm, w, d, ijk (grid order)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
    L = _ls_lib()
    n = L.orc_ls_band(ctypes.byref(g), _d(phi), float(eps), 0, None, None, None, None, None, None, None)
    xs = np.empty((n, 3))
    nrm = np.empty((n, 3))
    w = np.empty(n)
    d = np.empty(n)
    ijk = np.empty((n, 3), dtype=np.int32)
    curv = np.empty(n)
    sig2 = np.empty(n)
    L.orc_ls_band(ctypes.byref(g), _d(phi), float(eps), n, _d(xs), _d(nrm), _d(w), _d(d), ijk.ctypes.data_as(_I32),
                  _d(curv), _d(sig2))
    return {"xs": xs, "nrm": nrm, "w": w, "d": d, "ijk": ijk, "curv": curv, "sig2": sig2}


def solve_energy(xs, nrm, w, phys, z, q, eps_in, tol=1e-10, maxit=2000):
    """FP64 solve of the discrete system (Sec. 3.3, zero start) and its G_pol
    (Sec. 3.5): returns (p, G_pol in e^2/A, GMRES iterations)."""
    b = rhs(xs, nrm, z, q, eps_in)
    p, it, _, _ = gmres(xs, nrm, w, phys, b, tol=tol, maxit=maxit)
    return p, gpol(q, psi_rxn(xs, nrm, w, z, phys, p)), it


def extrapolated_energy(xs, nrm, w, phys, z, q, eps_in, tol=1e-10):
    """Richardson extrapolation of the tube regularisation (Sec. 2.2.1) to
    tau -> 0, reading its error as linear in tau: the system is solved with
    tau and with tau/2 on the same nodes and p* = 2 p(tau/2) - p(tau); G_pol is
    linear in p, so G* = 2 G(tau/2) - G(tau).  Returns (p*, G*, G(tau), G(tau/2))."""
    half = Phys(phys.eps_in, phys.eps_out, phys.kappa, 0.5 * phys.tau, phys.tube_rule)
    p1, g1, _ = solve_energy(xs, nrm, w, phys, z, q, eps_in, tol)
    p2, g2, _ = solve_energy(xs, nrm, w, half, z, q, eps_in, tol)
    return 2.0 * p2 - p1, 2.0 * g2 - g1, g1, g2


def jacobian(nodes):
    """Full Jacobian of the change of variables between Gamma and the level
    surface of d through each node (Sec. 2.2, reading: the last term is the sum
    of the 2x2 principal minors of the Hessian of d, so that J = (1 - d k1)(1 - d k2)
    in the level surface's principal curvatures k1, k2), clamped at 0 where the
    band is wider than a local radius of curvature."""
    d = nodes["d"]
    return np.maximum(1.0 - d * nodes["curv"] + d * d * nodes["sig2"], 0.0)


def jacobian_weights(nodes):
    """w_j = J_j delta_eps(d_j) h^3 from the J = 1 weights of the nodes."""
    return nodes["w"] * jacobian(nodes)


def ses_nodes(z, r, probe=1.4, h=0.5, eps=1.0):
    """Stages 1-2: band nodes of the solvent excluded surface of atoms (z, r)."""
    g, phi, _ = ls_ses(z, r, probe, h, eps)
    return ls_band(g, phi, eps)
