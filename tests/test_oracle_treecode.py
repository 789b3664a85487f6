"""Pins of the treecode oracle (oracle/treecode.py) to facts outside itself.

* Tensor-product Lagrange interpolation on Chebyshev points reproduces
  polynomials of degree n - 1 per axis and is the identity on its own points.
* Interpolating a parent cube's basis on a child cube's points is exact (the
  identity that lets a GPU build parent proxies from child proxies).
* The far-field kernels written as linear functions of the densities equal the
  C oracle's pair kernels (Sec. 2.2) for a single unit-normal source.
* With no far cluster the treecode is the direct operator.
* Every source tile is covered exactly once per target tile (near tile or
  inside exactly one far cluster).
* The error against the direct operator falls with the number of Chebyshev
  points and stays small.
"""
import numpy as np
import pytest

import oracle
from oracle import treecode as tc
from paper_1709_08070_gb300 import inputs

CENTRES = [(28.0 * i, 28.0 * j, 0.0) for i in range(3) for j in range(3)]


def _cloud(n_per=1000, radius=5.0, seed=4):
    return inputs.sphere_cluster_cloud(n_per, CENTRES, radius=radius, seed=seed)


def test_lagrange_reproduces_polynomials_and_is_identity_on_points():
    rng = np.random.default_rng(0)
    centre, half = np.array([1.5, -2.0, 0.25]), 3.0
    for n in (3, 4, 6):
        t = tc.proxy_points(centre, half, n)
        M = tc.interp_matrix(t, centre, half, n)
        np.testing.assert_allclose(M, np.eye(n ** 3), atol=1e-13)
        C = rng.standard_normal((n, n, n))  # coefficients of x^i y^j z^k, i, j, k < n

        def poly(P):
            u = (P - centre) / half
            V = [np.stack([u[:, a] ** e for e in range(n)], axis=1) for a in range(3)]
            return np.einsum("pi,pj,pk,ijk->p", V[0], V[1], V[2], C)

        y = centre + half * rng.uniform(-1.0, 1.0, size=(200, 3))
        interp = tc.interp_matrix(y, centre, half, n) @ poly(t)
        np.testing.assert_allclose(interp, poly(y), rtol=0, atol=1e-11 * np.abs(poly(y)).max())


def test_child_to_parent_transfer_is_exact():
    rng = np.random.default_rng(1)
    n = 6
    pc, ph = np.zeros(3), 4.0
    cc, chh = np.array([1.0, -1.5, 0.5]), 1.7
    y = cc + chh * rng.uniform(-1.0, 1.0, size=(50, 3))
    tchild = tc.proxy_points(cc, chh, n)
    direct = tc.interp_matrix(y, pc, ph, n)  # L^p_l(y)
    via = tc.interp_matrix(y, cc, chh, n) @ tc.interp_matrix(tchild, pc, ph, n)
    np.testing.assert_allclose(via, direct, rtol=0, atol=1e-12)


def test_far_kernels_match_pair_kernels_for_unit_sources():
    rng = np.random.default_rng(2)
    for kappa, eps_in in ((0.1257, 2.0), (0.0, 1.0), (0.5, 4.0)):
        P = oracle.Phys(eps_in, 80.0, kappa, 0.3)
        x = rng.standard_normal((3, 3)) * 2.0
        nx = rng.standard_normal((3, 3))
        nx /= np.linalg.norm(nx, axis=1, keepdims=True)
        y = x[0] + np.array([6.0, 1.0, -2.0]) + rng.standard_normal((4, 3))
        m = rng.standard_normal((4, 3))
        m /= np.linalg.norm(m, axis=1, keepdims=True)
        a, b = rng.uniform(-1, 1, 4), rng.uniform(-1, 1, 4)
        f1, f2 = tc.far_kernels(x, nx, y, a[:, None] * m, b, P)
        for i in range(3):
            e1 = e2 = 0.0
            for j in range(4):
                K, tube = oracle.pair_kernels(x[i], nx[i], y[j], m[j], P)
                assert not tube
                e1 += K[0] * a[j] - K[1] * b[j]
                e2 += K[2] * a[j] - K[3] * b[j]
            np.testing.assert_allclose([f1[i], f2[i]], [e1, e2], rtol=1e-12, atol=1e-15)


def test_no_far_cluster_is_the_direct_operator():
    xs, nr, w = _cloud(n_per=400)
    N = xs.shape[0]
    P = oracle.Phys(2.0, 80.0, 0.1257, 0.3)
    p = inputs.random_vector(2 * N, seed=3)
    tree = tc.TileTree(xs)
    lists = tree.lists(1e-9, 0.3)
    assert tc.list_sizes(lists)[1] == 0
    y = tc.treecode_matvec(xs, nr, w, P, p, tree=tree, lists=lists)
    ye = oracle.matvec(xs, nr, w, P, p)
    np.testing.assert_allclose(y, ye, rtol=0, atol=1e-13 * np.abs(ye).max())


def test_every_source_tile_once_per_target_tile():
    xs, nr, w = _cloud(n_per=1000)
    tree = tc.TileTree(xs)
    tiles = set(range(tree.n_s))
    for theta in (0.4, 0.7, 1.0):
        lists = tree.lists(theta, 0.3)
        assert tc.list_sizes(lists)[1] > 0
        for near, far in lists:
            seen = list(near)
            for ci in far:
                c = tree.clusters[ci]
                assert c.j0 % tree.stile == 0
                seen += list(range(c.j0 // tree.stile, -(-c.j1 // tree.stile)))
            assert sorted(seen) == sorted(tiles)


def test_far_clusters_keep_proxies_out_of_the_tube():
    xs, nr, w = _cloud(n_per=1000)
    tree = tc.TileTree(xs)
    tau = 0.4
    fd = max(2 * tau, 1.5) * 1.001 + 1e-3
    for t, (near, far) in enumerate(tree.lists(0.8, tau)):
        tx = xs[t * tree.ttile:min((t + 1) * tree.ttile, tree.N)]
        for ci in far:
            c = tree.clusters[ci]
            pr = tc.proxy_points(c.centre, c.half, 6)
            dmin = np.sqrt(((tx[:, None, :] - pr[None, :, :]) ** 2).sum(-1)).min()
            assert dmin >= fd


@pytest.mark.parametrize("theta", [0.6])
def test_error_falls_with_the_chebyshev_order(theta):
    xs, nr, w = _cloud(n_per=1000)
    N = xs.shape[0]
    P = oracle.Phys(2.0, 80.0, 0.1257, 0.3)
    p = inputs.random_vector(2 * N, seed=1)
    ye = oracle.matvec(xs, nr, w, P, p)
    tree = tc.TileTree(xs)
    lists = tree.lists(theta, 0.3)
    assert tc.list_sizes(lists)[1] > 0
    errs = []
    for n in (3, 4, 6):
        y = tc.treecode_matvec(xs, nr, w, P, p, n=n, tree=tree, lists=lists)
        errs.append(max(np.linalg.norm(y[:N] - ye[:N]) / np.linalg.norm(ye[:N]),
                        np.linalg.norm(y[N:] - ye[N:]) / np.linalg.norm(ye[N:])))
    print("treecode error vs direct, theta %.1f, n = 3, 4, 6: %s" % (theta, ["%.2e" % e for e in errs]))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-7


def test_cubes_nest_and_hold_their_nodes():
    xs, nr, w = _cloud(n_per=700)
    tree = tc.TileTree(xs)
    for c in tree.clusters:
        seg = xs[c.j0:c.j1]
        assert np.all(np.abs(seg - c.centre) <= c.half * (1 + 1e-12))
        for ci in c.children:
            q = tree.clusters[ci]
            assert np.all(np.abs(q.centre - c.centre) + q.half <= c.half * (1 + 1e-12))


def test_far_fields_equal_far_kernels_for_any_target_normal():
    rng = np.random.default_rng(7)
    for kappa, eps_in in ((0.1257, 2.0), (0.0, 1.0)):
        P = oracle.Phys(eps_in, 80.0, kappa, 0.3)
        s = rng.standard_normal((5, 3))
        nx = rng.standard_normal((5, 3))
        nx /= np.linalg.norm(nx, axis=1, keepdims=True)
        t = np.array([7.0, -2.0, 3.0]) + rng.standard_normal((6, 3))
        d, beta = rng.standard_normal((6, 3)), rng.standard_normal(6)
        f1, f2 = tc.far_kernels(s, nx, t, d, beta, P)
        g1, V = tc.far_fields(s, t, d, beta, P)
        np.testing.assert_allclose(g1, f1, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(np.einsum("ik,ik->i", nx, V), f2, rtol=1e-12, atol=1e-16)


def test_target_interpolation_clears_the_tube_and_stays_accurate():
    xs, nr, w = _cloud(n_per=1000)
    N = xs.shape[0]
    tau = 0.3
    P = oracle.Phys(2.0, 80.0, 0.1257, tau)
    p = inputs.random_vector(2 * N, seed=1)
    ye = oracle.matvec(xs, nr, w, P, p)
    tree = tc.TileTree(xs)
    fd = max(2 * tau, 1.5) * 1.001 + 1e-3
    lists = tree.lists(0.8, tau, interp=True)
    sizes = tc.list_sizes(lists)
    assert sizes[2] > 0
    for t, (near, far, fint) in enumerate(lists):
        sp = tc.proxy_points(tree.t_centre[t], tree.t_half[t], 6)
        tx = xs[t * tree.ttile:min((t + 1) * tree.ttile, tree.N)]
        assert np.all(np.abs(tx - tree.t_centre[t]) <= tree.t_half[t] * (1 + 1e-12))
        for ci in fint:
            c = tree.clusters[ci]
            pr = tc.proxy_points(c.centre, c.half, 6)
            assert np.sqrt(((sp[:, None, :] - pr[None, :, :]) ** 2).sum(-1)).min() >= fd
    errs = []
    for n in (4, 6):
        y = tc.treecode_matvec(xs, nr, w, P, p, n=n, tree=tree, lists=lists)
        errs.append(max(np.linalg.norm(y[:N] - ye[:N]) / np.linalg.norm(ye[:N]),
                        np.linalg.norm(y[N:] - ye[N:]) / np.linalg.norm(ye[N:])))
    y0 = tc.treecode_matvec(xs, nr, w, P, p, n=6, tree=tree, lists=tree.lists(0.8, tau))
    e0 = max(np.linalg.norm(y0[:N] - ye[:N]) / np.linalg.norm(ye[:N]),
             np.linalg.norm(y0[N:] - ye[N:]) / np.linalg.norm(ye[N:]))
    print("target interpolation, theta 0.8, lists %s: error n = 4, 6: %s (source side only: %.2e)"
          % (sizes, ["%.2e" % e for e in errs], e0))
    assert errs[0] > errs[1] and errs[1] < 5.0 * e0 + 1e-9 and errs[1] < 1e-6


@pytest.mark.parametrize("theta,n_per,interp,order,bound", [(0.6, 1000, 1, 6, 5e-7), (0.7, 1000, 0, 5, 5e-7),
                                                            (0.8, 1500, 1, 4, 1e-5)])
def test_error_within_the_documented_bound(theta, n_per, interp, order, bound):
    """The approximation bound the GPU tests hold both treecodes to (relative
    2-norm and worst element / max |y| per output block against the direct
    operator, theta <= 0.8): 5e-7 with 5 or 6 Chebyshev points per axis,
    1e-5 with 4.  It depends on the interpolation order and the separation
    only, not on how nodes are grouped into tiles."""
    xs, nr, w = _cloud(n_per)
    N = xs.shape[0]
    P = oracle.Phys(2.0, 80.0, 0.1257, 0.3)
    p = inputs.random_vector(2 * N, seed=6)
    tree = tc.TileTree(xs)
    lists = tree.lists(theta, 0.3, bool(interp))
    yt = tc.treecode_matvec(xs, nr, w, P, p, n=order, tree=tree, lists=lists)
    ye = oracle.matvec(xs, nr, w, P, p)
    for blk in (slice(0, N), slice(N, 2 * N)):
        assert np.linalg.norm(yt[blk] - ye[blk]) / np.linalg.norm(ye[blk]) < bound
        assert np.max(np.abs(yt[blk] - ye[blk])) / np.max(np.abs(ye[blk])) < bound
