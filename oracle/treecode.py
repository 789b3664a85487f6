"""Treecode form of the IBIM operator (test infrastructure only).

The far field of K W p (Sec. 2.2, discrete system) is approximated by source-side
Chebyshev interpolation, in the manner of the paper's far-field accelerator (a
black-box FMM built on Chebyshev interpolation, Sec. 4): the densities of a
cluster of sources are transferred onto a tensor grid of Chebyshev points of its
bounding cube ("proxies"), and a target far from the cluster interacts with the
proxies instead of the sources.  There are no local expansions: the proxy
interactions are evaluated directly (a barycentric Lagrange treecode).  Near
sources are summed exactly, with the tube rule, as in the direct operator.

Interpolating the densities is valid because every kernel is linear in the
source's density pair: with d_j = a_j m_j (a vector) and b_j (a scalar),
a_j = w_j psi_j, b_j = w_j psin_j,
    K11 a_j = s_d (1 - th1 A) / (4 pi rho^3),          s_d = r . d_j
    K12 b_j = (1 - E) / (4 pi rho) b_j
    K21 a_j = [(1 - A) c_d - (3 - B) s_x s_d / rho^2] / (4 pi rho^3),  c_d = n_x . d_j
    K22 b_j = -s_x (1 - th2 A) / (4 pi rho^3) b_j
so the sum over a cluster is a sum of kernels of the positions alone times the
densities, and the densities can be moved onto proxy points.

Structure (the tiling is chosen so that a GPU can stream proxies like sources):
  * source tiles of 256 consecutive nodes; clusters are contiguous node ranges
    split as a coordinate bisection of the node order splits them: a range of
    n > 256 nodes into a left part of B max(1, round(n / 2B)) nodes, B = 1024
    for n >= 2048 and 256 otherwise, down to single tiles (for nodes ordered by
    that bisection every cluster is one of its ranges);
  * proxy cube of a cluster: the smallest axis box holding its nodes and its
    children's cubes, made a cube about the box centre with the largest half
    extent (at least kMinHalf) as half side, so every cube lies inside its
    parent's; n^3 Chebyshev points of the second kind, radius = half side x
    sqrt(3);
  * target tiles of 512 consecutive nodes, bounding box centre and
    half-diagonal r_T;
  * a cluster is far from a target tile when r_T + r_C <= theta D and
    D >= far_dist + r_T + r_C + kFarMargin (D the distance of the centres,
    far_dist = max(2 tau_max, 1.5) 1.001 + 1e-3): every target-proxy distance
    is then at least far_dist, so no proxy lies in the regularisation tube
    (Sec. 2.2.1) and the kernels need no near-field care;
  * lists by depth-first traversal from the root: far clusters take proxies,
    a one-tile cluster that is not far is summed directly;
  * target-side interpolation (optional): a far cluster that is also far from
    the target tile's own proxy cube (radius r_Tc = half side x sqrt(3):
    r_Tc + r_C <= theta D and D >= far_dist + r_Tc + r_C + kFarMargin) is
    evaluated at the tile's n^3 target proxies instead of its targets.  y1 is
    a scalar function of the target position and y2 = n_x . V(x) with the
    vector field
        V = [g d - (3 - B) (r.d / rho^2) r + (1 - th2 A) b r] / (4 pi rho^3),
    g = 1 - A, so the four fields (y1, V) are interpolated from the target
    proxies to the targets with the same tensor-product Lagrange basis.

Parity: pinned by polynomial reproduction of the interpolation, the
child-to-parent transfer identity, agreement with the direct operator when no
cluster is far, convergence in n, and coverage of every source tile exactly
once per target tile (tests/test_oracle_treecode.py).
"""
import math

import numpy as np

from . import oracle as _orc

kMinHalf = 1e-3   # smallest proxy-cube half side (A)
kFarMargin = 0.25  # extra gap of a far cluster (A)


def cheb_points(n):
    """Chebyshev points of the second kind on [-1, 1] and their barycentric weights."""
    k = np.arange(n)
    pts = np.cos(np.pi * k / (n - 1))
    wts = np.where(k % 2 == 0, 1.0, -1.0)
    wts[0] *= 0.5
    wts[-1] *= 0.5
    return pts, wts


def lagrange_1d(y, centre, half, n):
    """L[j, k] = l_k(y_j), the Lagrange basis of the n Chebyshev points of
    [centre - half, centre + half] at the coordinates y (barycentric form;
    a coordinate on a point gives the unit vector)."""
    pts, wts = cheb_points(n)
    t = centre + half * pts
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    diff = y[:, None] - t[None, :]
    hit = diff == 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        q = wts[None, :] / diff
        L = q / q.sum(axis=1, keepdims=True)
    rows = hit.any(axis=1)
    if rows.any():
        L[rows] = hit[rows].astype(np.float64)
    return L


def proxy_points(centre, half, n):
    """The n^3 proxies of a cube, proxy k = (kx n + ky) n + kz."""
    pts, _ = cheb_points(n)
    g = [centre[a] + half * pts for a in range(3)]
    X, Y, Z = np.meshgrid(g[0], g[1], g[2], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def interp_matrix(ys, centre, half, n):
    """M[j, k] = L_k(y_j) for the tensor-product basis of a cube."""
    Lx = lagrange_1d(ys[:, 0], centre[0], half, n)
    Ly = lagrange_1d(ys[:, 1], centre[1], half, n)
    Lz = lagrange_1d(ys[:, 2], centre[2], half, n)
    return (Lx[:, :, None, None] * Ly[:, None, :, None] * Lz[:, None, None, :]).reshape(ys.shape[0], -1)


class Cluster:
    __slots__ = ("j0", "j1", "children", "centre", "half", "radius")


def split_point(n):
    """Size of the left part of a cluster of n > 256 nodes."""
    B = 1024 if n >= 2048 else 256
    return B * max(1, int(math.floor(n / (2.0 * B) + 0.5)))


def target_cube(centre, half_extent):
    """Proxy cube of a target tile: about its box centre, the largest half
    extent (at least kMinHalf) as half side."""
    return centre, max(max(half_extent[0], half_extent[1], half_extent[2]), kMinHalf)


class TileTree:
    """Clusters of source tiles and the target tiles of an ordered node set."""

    stile, ttile = 256, 512

    def __init__(self, xs):
        xs = np.ascontiguousarray(xs, dtype=np.float64).reshape(-1, 3)
        self.xs, self.N = xs, xs.shape[0]
        stile, ttile = self.stile, self.ttile
        self.n_s = -(-self.N // stile)
        self.clusters = []
        self._make(0, self.N)
        self.n_t = -(-self.N // ttile)
        self.t_centre = np.zeros((self.n_t, 3))
        self.t_radius = np.zeros(self.n_t)
        self.t_half = np.zeros(self.n_t)    # target proxy cube half side
        self.t_cradius = np.zeros(self.n_t)  # its half-diagonal
        for t in range(self.n_t):
            mn, mx = self._box(t * ttile, min((t + 1) * ttile, self.N))
            self.t_centre[t] = 0.5 * (mn + mx)
            e = 0.5 * (mx - mn)
            self.t_radius[t] = math.sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2])
            _, self.t_half[t] = target_cube(self.t_centre[t], e)
            self.t_cradius[t] = math.sqrt(3.0 * self.t_half[t] * self.t_half[t])

    def _box(self, j0, j1):
        seg = self.xs[j0:j1]
        return seg.min(axis=0), seg.max(axis=0)

    def _make(self, j0, j1):
        c = Cluster()
        c.j0, c.j1, c.children = j0, j1, ()
        idx = len(self.clusters)
        self.clusters.append(c)
        if j1 - j0 > self.stile:
            k = split_point(j1 - j0)
            c.children = (self._make(j0, j0 + k), self._make(j0 + k, j1))
        mn, mx = self._box(j0, j1)
        mn, mx = [float(v) for v in mn], [float(v) for v in mx]
        for ci in c.children:
            q = self.clusters[ci]
            for a in range(3):
                mn[a] = min(mn[a], q.centre[a] - q.half)
                mx[a] = max(mx[a], q.centre[a] + q.half)
        c.centre = np.array([0.5 * (mn[a] + mx[a]) for a in range(3)])
        e = [0.5 * (mx[a] - mn[a]) for a in range(3)]
        c.half = max(max(e[0], e[1], e[2]), kMinHalf)
        c.radius = math.sqrt(3.0 * c.half * c.half)
        return idx

    def far(self, t, ci, theta, far_dist):
        c = self.clusters[ci]
        d = self.t_centre[t] - c.centre
        D = math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
        rT = self.t_radius[t]
        return (rT + c.radius <= theta * D) and (D >= far_dist + rT + c.radius + kFarMargin)

    def far_interp(self, t, ci, theta, far_dist):
        """Far also from the target tile's proxy cube (target-side interpolation)."""
        c = self.clusters[ci]
        d = self.t_centre[t] - c.centre
        D = math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
        rT = self.t_cradius[t]
        return (rT + c.radius <= theta * D) and (D >= far_dist + rT + c.radius + kFarMargin)

    def lists(self, theta, tau_max, interp=False):
        """Per target tile: (near source tiles, far clusters), depth-first order;
        with interp, (near, far, far_interp): far clusters that pass the target
        cube's test go to far_interp instead of far."""
        fd = max(2.0 * tau_max, 1.5) * 1.001 + 1e-3
        out = []
        for t in range(self.n_t):
            near, far, fint = [], [], []
            stack = [0]
            while stack:
                ci = stack.pop()
                c = self.clusters[ci]
                if self.far(t, ci, theta, fd):
                    if interp and self.far_interp(t, ci, theta, fd):
                        fint.append(ci)
                    else:
                        far.append(ci)
                elif not c.children:
                    near.append(c.j0 // self.stile)
                else:
                    stack.append(c.children[1])
                    stack.append(c.children[0])
            out.append((near, far, fint) if interp else (near, far))
        return out


def far_kernels(x, nx, t, d, beta, phys):
    """Contributions (y1, y2) of proxies at t with vector densities d and scalar
    densities beta to targets x with normals nx (the four kernels of Sec. 2.2
    written as linear functions of the source densities; no tube: far only).
    x, nx: (m, 3); t, d: (p, 3); beta: (p,).  Returns two (m,) arrays."""
    r = x[:, None, :] - t[None, :, :]
    rho2 = np.einsum("ijk,ijk->ij", r, r)
    rho = np.sqrt(rho2)
    s_x = np.einsum("ijk,ik->ij", r, nx)
    s_d = np.einsum("ijk,jk->ij", r, d)
    c_d = nx @ d.T
    kap = phys.kappa
    E = np.exp(-kap * rho)
    A = E * (1.0 + kap * rho)
    B = E * (3.0 + 3.0 * kap * rho + kap * kap * rho2)
    th1 = phys.eps_out / phys.eps_in
    th2 = phys.eps_in / phys.eps_out
    fp = 4.0 * np.pi
    rho3 = rho2 * rho
    k11 = s_d * (1.0 - th1 * A) / (fp * rho3)
    k12 = (1.0 - E) / (fp * rho)
    k21 = (c_d * (1.0 - A) - (3.0 - B) * s_x * s_d / rho2) / (fp * rho3)
    k22 = -s_x * (1.0 - th2 * A) / (fp * rho3)
    y1 = (k11 - k12 * beta[None, :]).sum(axis=1)
    y2 = (k21 - k22 * beta[None, :]).sum(axis=1)
    return y1, y2


def far_fields(s, t, d, beta, phys):
    """The fields (y1, V) at points s of proxies at t with densities (d, beta):
    y1 as in far_kernels and V with y2 = n_x . V (Sec. 2.2 kernels, linear in
    the target normal).  Returns (m,) and (m, 3)."""
    r = s[:, None, :] - t[None, :, :]
    rho2 = np.einsum("ijk,ijk->ij", r, r)
    rho = np.sqrt(rho2)
    s_d = np.einsum("ijk,jk->ij", r, d)
    kap = phys.kappa
    E = np.exp(-kap * rho)
    A = E * (1.0 + kap * rho)
    B = E * (3.0 + 3.0 * kap * rho + kap * kap * rho2)
    th1 = phys.eps_out / phys.eps_in
    th2 = phys.eps_in / phys.eps_out
    fp = 4.0 * np.pi
    rho3 = rho2 * rho
    y1 = (s_d * (1.0 - th1 * A) / (fp * rho3) - (1.0 - E) / (fp * rho) * beta[None, :]).sum(axis=1)
    coef = (-(3.0 - B) * s_d / rho2 + (1.0 - th2 * A) * beta[None, :]) / (fp * rho3)
    V = np.einsum("ij,jk->ik", (1.0 - A) / (fp * rho3), d) + np.einsum("ij,ijk->ik", coef, r)
    return y1, V


def cluster_densities(tree, ci, nrm, a, b, n):
    """Proxy densities of cluster ci: (proxies (n^3, 3), D (n^3, 3), beta (n^3,)),
    D_k = sum_j L_k(y_j) a_j m_j and beta_k = sum_j L_k(y_j) b_j over its nodes."""
    c = tree.clusters[ci]
    j0, j1 = c.j0, c.j1
    M = interp_matrix(tree.xs[j0:j1], c.centre, c.half, n)
    D = M.T @ (a[j0:j1, None] * nrm[j0:j1])
    beta = M.T @ b[j0:j1]
    return proxy_points(c.centre, c.half, n), D, beta


def treecode_matvec(xs, nrm, w, phys, p, theta=0.5, n=6, tau_max=None, tree=None, lists=None, interp=False):
    """(Lambda + K W) p with the far field of every target tile taken from the
    proxies of its far clusters and the rest summed exactly (tube rule
    included) by the direct oracle; with interp, the far clusters that pass
    the target cube's test act on the tile's target proxies and their fields
    are interpolated to the targets."""
    xs, nrm, w = _orc._geom(xs, nrm, w)
    N = w.shape[0]
    p = _orc._f64(p, 2 * N)
    tau_max = phys.tau if tau_max is None else tau_max
    if tree is None:
        tree = TileTree(xs)
    stile, ttile = tree.stile, tree.ttile
    if lists is None:
        lists = tree.lists(theta, tau_max, interp)
    a = w * p[:N]
    b = w * p[N:]
    cache = {}
    y = np.empty(2 * N)
    for t, entry in enumerate(lists):
        near, far = entry[0], entry[1]
        fint = entry[2] if len(entry) > 2 else []
        i0, i1 = t * ttile, min((t + 1) * ttile, N)
        rows = np.arange(i0, i1)
        wn = np.zeros(N)
        for s in near:
            wn[s * stile:min((s + 1) * stile, N)] = w[s * stile:min((s + 1) * stile, N)]
        y1, y2 = _orc.matvec_rows(xs, nrm, wn, phys, p, rows)  # Lambda p + near sums
        for ci in far:
            if ci not in cache:
                cache[ci] = cluster_densities(tree, ci, nrm, a, b, n)
            tp, D, beta = cache[ci]
            f1, f2 = far_kernels(xs[i0:i1], nrm[i0:i1], tp, D, beta, phys)
            y1 = y1 + f1
            y2 = y2 + f2
        if fint:
            th = tree.t_half[t]
            sp = proxy_points(tree.t_centre[t], th, n)
            F1 = np.zeros(sp.shape[0])
            FV = np.zeros((sp.shape[0], 3))
            for ci in fint:
                if ci not in cache:
                    cache[ci] = cluster_densities(tree, ci, nrm, a, b, n)
                tp, D, beta = cache[ci]
                g1, gV = far_fields(sp, tp, D, beta, phys)
                F1 += g1
                FV += gV
            M = interp_matrix(xs[i0:i1], tree.t_centre[t], th, n)
            y1 = y1 + M @ F1
            y2 = y2 + np.einsum("ik,ik->i", nrm[i0:i1], M @ FV)
        y[i0:i1] = y1
        y[N + i0:N + i1] = y2
    return y


def list_sizes(lists):
    """(near source tiles, far clusters[, far clusters by interpolation]) summed over target tiles."""
    return tuple(sum(len(e[k]) for e in lists) for k in range(len(lists[0])))
