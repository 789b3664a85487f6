"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these checks compares the oracle with itself: kernels are checked
against finite differences of the fundamental solutions, the tube value
against numerical quadrature, band extraction against the paper's printed
node counts, whole solves against the Born and Kirkwood closed forms and the
paper's Table 2 errors, GMRES against a dense LU solve.
"""
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from oracle import closed_forms as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _G(x, y, kappa):
    """Fundamental solution e^{-kappa |x-y|}/(4 pi |x-y|) (Sec. 2.1), written out here."""
    r = np.linalg.norm(np.asarray(x) - np.asarray(y))
    return np.exp(-kappa * r) / (4 * np.pi * r)


def _D(x, y, kappa):
    """G0 - Gk = (1 - e^{-kappa r})/(4 pi r), written with expm1 so that it keeps
    full relative accuracy (its derivatives are what K21 differentiates)."""
    r = np.linalg.norm(np.asarray(x) - np.asarray(y))
    return -np.expm1(-kappa * r) / (4 * np.pi * r)


def _fd_kernels(x, nx, y, ny, eps_in, eps_out, kappa):
    """K11, K12, K21, K22 from central differences of G0, Gk and G0 - Gk along
    the normals, Richardson-extrapolated (steps h and h/2)."""
    def dny(F, xx, yy, hs):
        return (F(xx, yy + hs * ny) - F(xx, yy - hs * ny)) / (2 * hs)

    def dnx(F, xx, yy, hs):
        return (F(xx + hs * nx, yy) - F(xx - hs * nx, yy)) / (2 * hs)

    def dnxdny(F, hs):
        return (dny(F, x + hs * nx, y, hs) - dny(F, x - hs * nx, y, hs)) / (2 * hs)

    def rich(f, hs):
        return (4.0 * f(hs / 2) - f(hs)) / 3.0

    G0 = lambda a, b: _G(a, b, 0.0)
    Gk = lambda a, b: _G(a, b, kappa)
    D = lambda a, b: _D(a, b, kappa)
    th1, th2 = eps_out / eps_in, eps_in / eps_out
    h1 = 1e-3
    K11 = rich(lambda hs: dny(G0, x, y, hs) - th1 * dny(Gk, x, y, hs), h1)
    K12 = D(x, y)
    K21 = rich(lambda hs: dnxdny(D, hs), h1)
    K22 = rich(lambda hs: dnx(G0, x, y, hs) - th2 * dnx(Gk, x, y, hs), h1)
    return np.array([K11, K12, K21, K22])


@pytest.mark.parametrize("kappa", [0.0, 0.1257, 0.2, 1.3])
def test_kernels_match_finite_differences(kappa):
    rng = np.random.default_rng(7)
    P = oracle.Phys(2.0, 80.0, kappa, tau=0.1)
    for _ in range(40):
        x = rng.uniform(-3, 3, 3)
        y = rng.uniform(-3, 3, 3)
        if np.linalg.norm(x - y) < 0.5:
            continue
        nx = rng.standard_normal(3)
        nx /= np.linalg.norm(nx)
        ny = rng.standard_normal(3)
        ny /= np.linalg.norm(ny)
        K, tube = oracle.pair_kernels(x, nx, y, ny, P)
        assert not tube
        Kfd = _fd_kernels(x, nx, y, ny, P.eps_in, P.eps_out, kappa)
        # absolute floor: FD rounding, eps_mach * |G| / step^2 ~ 1e-11
        assert np.all(np.abs(K - Kfd) <= 1e-6 * np.abs(Kfd) + 2e-11), (K, Kfd)


def test_hypersingular_difference_is_order_one_over_r():
    """Sec. 2.1: the K21 combination is O(1/|x-y|) as |x-y| -> 0."""
    P = oracle.Phys(1.0, 80.0, 0.1257, tau=1e-9, tube_rule=1)
    n = np.array([0.0, 0.0, 1.0])
    vals = []
    for rho in (1e-1, 1e-2, 1e-3):
        K, _ = oracle.pair_kernels(np.array([rho, 0, 0]), n, np.zeros(3), n, P)
        vals.append(K[2] * rho)
    vals = np.array(vals)
    assert np.all(np.isfinite(vals))
    assert np.max(np.abs(vals)) / np.min(np.abs(vals)) < 1.2


@pytest.mark.parametrize("kappa,tau", [(0.1257, 0.25), (0.2, 0.125), (1.0, 0.5)])
def test_tube_value_of_K12_is_disc_average(kappa, tau):
    """Sec. 2.2.1: inside the tube K12 is the average of G0 - Gk over the tangent disc."""
    P = oracle.Phys(1.0, 80.0, kappa, tau=tau)
    n = np.array([0.0, 0.0, 1.0])
    K, tube = oracle.pair_kernels(np.zeros(3), n, np.zeros(3), n, P)  # self pair
    assert tube
    f = lambda s: (1.0 - np.exp(-kappa * s)) / (4 * np.pi * s) * 2 * np.pi * s
    avg = integrate.quad(f, 0.0, tau, epsabs=1e-14, epsrel=1e-13)[0] / (np.pi * tau * tau)
    assert K[1] == pytest.approx(avg, rel=1e-10)
    assert K[0] == 0.0 and K[2] == 0.0 and K[3] == 0.0


def test_kappa_zero_limits():
    """Sec. 2.1: at kappa = 0, K12 vanishes (tube and off-tube) and the system decouples."""
    P = oracle.Phys(1.0, 80.0, 0.0, tau=0.25)
    n = np.array([0.0, 0.0, 1.0])
    K, tube = oracle.pair_kernels(np.zeros(3), n, np.zeros(3), n, P)
    assert tube and K[1] == 0.0
    K, tube = oracle.pair_kernels(np.array([1.0, 0.3, 0.2]), n, np.zeros(3), n, P)
    assert not tube and K[1] == 0.0
    g = oracle.sphere_nodes(1.5, h=0.25, eps=0.5)
    N = g["w"].size
    p = np.random.default_rng(1).standard_normal(2 * N)
    p2 = p.copy()
    p2[N:] = np.random.default_rng(2).standard_normal(N)
    y = oracle.matvec(g["xs"], g["nrm"], g["w"], P, p)
    y2 = oracle.matvec(g["xs"], g["nrm"], g["w"], P, p2)
    np.testing.assert_array_equal(y[:N], y2[:N])  # psi rows blind to psi_n


def test_equal_dielectrics_no_screening_has_no_reaction_field():
    """eps_I = eps_E and kappa = 0: every kernel vanishes, G_pol = 0."""
    P = oracle.Phys(2.0, 2.0, 0.0, tau=0.25)
    g = oracle.sphere_nodes(2.0, h=0.25, eps=0.5)
    z = np.array([[0.3, -0.2, 0.1], [0.0, 0.5, -0.4]])
    q = np.array([1.0, -0.5])
    b = oracle.rhs(g["xs"], g["nrm"], z, q, 2.0)
    A = oracle.matvec(g["xs"], g["nrm"], g["w"], P, b)
    np.testing.assert_allclose(A, b, rtol=0, atol=1e-15 * np.max(np.abs(b)))
    psi = oracle.psi_rxn(g["xs"], g["nrm"], g["w"], z, P, b)
    assert np.max(np.abs(psi)) < 1e-15


def test_tube_rule_geometry():
    """Tangent-plane distance test (Sec. 2.2.1) and the |r| < 2 tau reading."""
    n = np.array([0.0, 0.0, 1.0])
    tau = 0.5
    for rule in (0, 1):
        P = oracle.Phys(1.0, 80.0, 0.1257, tau=tau, tube_rule=rule)
        assert oracle.pair_kernels(np.zeros(3), n, np.array([0.45, 0, 0]), n, P)[1]
        assert not oracle.pair_kernels(np.zeros(3), n, np.array([0.55, 0, 0]), n, P)[1]
        assert oracle.pair_kernels(np.zeros(3), n, np.array([0.0, 0.1, -0.9]), n, P)[1]
        far = oracle.pair_kernels(np.zeros(3), n, np.array([0.0, 0.1, -3.0]), n, P)[1]
        assert far == (rule == 1)


def test_delta_eps_moments():
    """Sec. 3.2 cosine weight: unit mass, even, compact support, second moment
    eps^2 (1/3 - 2/pi^2)."""
    eps = 0.7
    f = lambda t: oracle.delta_eps(t, eps)
    assert integrate.quad(f, -eps, eps, epsabs=1e-13)[0] == pytest.approx(1.0, abs=1e-12)
    assert integrate.quad(lambda t: t * f(t), -eps, eps, epsabs=1e-13)[0] == pytest.approx(0.0, abs=1e-13)
    m2 = integrate.quad(lambda t: t * t * f(t), -eps, eps, epsabs=1e-14)[0]
    assert m2 == pytest.approx(eps * eps * (1 / 3 - 2 / np.pi ** 2), rel=1e-10)
    assert f(eps) == 0.0 and f(-eps) == 0.0 and f(1.2 * eps) == 0.0
    assert f(0.3) == pytest.approx(f(-0.3), rel=0, abs=0)


def _table2():
    rows = []
    with open(os.path.join(GOLDEN, "table2_single_ion.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows.append((int(v[0]), float(v[1]), int(v[2]), int(v[3]), float(v[4]),
                             float(v[5]), float(v[6])))
    return rows


@pytest.mark.parametrize("n", [64, 128, 256])
def test_band_node_count_matches_table2(n):
    """Sec. 4.2 Table 2 D.O.F.: band {|d| < 2h} of the unit sphere on the
    [-1.5, 1.5]^3 grid with n^3 cells."""
    dof = {r[0]: r[2] for r in _table2()}[n]
    h = 3.0 / n
    g = oracle.sphere_nodes(1.0, h=h, eps=2 * h)
    assert g["w"].size == dof


def test_sphere_area_closed_form():
    """Sec. 3.4 area with J = 1 on a sphere: 4 pi (R^2 + c eps^2) + O(h^2),
    c = 1/3 - 2/pi^2 the weight's second moment (Sec. 3.2)."""
    for R, h, k in ((2.0, 0.25, 3), (2.0, 0.125, 2), (5.0, 0.25, 2)):
        eps = k * h
        A = oracle.area(oracle.sphere_nodes(R, h=h, eps=eps)["w"])
        ref = 4 * np.pi * (R * R + (1 / 3 - 2 / np.pi ** 2) * eps * eps)
        assert abs(A / ref - 1) < 2e-4, (R, h, A, ref)


def test_area_error_column_of_table2():
    """Table 2 area error (1.24e-3 at 64^3, 2.88e-4 at 128^3) to within 15%."""
    for n, tk, dof, it, sol, aerr, eerr in _table2():
        if n > 128 or tk != 1.0:
            continue
        h = 3.0 / n
        A = oracle.area(oracle.sphere_nodes(1.0, h=h, eps=2 * h)["w"])
        assert abs(abs(A / (4 * np.pi) - 1) / aerr - 1) < 0.15


def test_gauss_double_layer_identity():
    """Sec. 2.1 kernel dG0/dn(y): on a sphere the integral over the surface
    is -1/2; without the tube cap (tangent radius tau) it is
    -1/2 + 1/2 sin(arcsin(tau/R)/2).  The IBIM sum with J = 1 carries the
    area factor (1 + c eps^2/R^2)."""
    R, h, k, tau = 3.0, 0.25, 2, 0.25
    eps = k * h
    g = oracle.sphere_nodes(R, h=h, eps=eps)
    N = g["w"].size
    # eps_E/eps_I = 1, kappa large: K11 = dG0/dn(y) - e^{-kappa rho}(...) = dG0/dn(y) off the tube
    P = oracle.Phys(1.0, 1.0, 400.0, tau=tau)
    p = np.concatenate([np.ones(N), np.zeros(N)])
    rows = np.arange(0, N, max(1, N // 300))
    y1, _ = oracle.matvec_rows(g["xs"], g["nrm"], g["w"], P, p, rows)
    S = y1 - 1.0  # lambda1 = 1
    c = 1 / 3 - 2 / np.pi ** 2
    ref = (-0.5 + 0.5 * np.sin(0.5 * np.arcsin(tau / R))) * (1 + c * eps * eps / (R * R))
    assert abs(np.mean(S) / ref - 1) < 3e-3
    assert np.max(np.abs(S / ref - 1)) < 3e-2


def test_gmres_matches_dense_lu():
    """Brute force on a tiny input: GMRES vs LU of the dense 2N x 2N matrix."""
    g = oracle.sphere_nodes(1.0, h=0.25, eps=0.5)
    N = g["w"].size
    assert N < 1000
    P = oracle.Phys(1.0, 80.0, 0.1257, tau=0.25)
    A = oracle.dense(g["xs"], g["nrm"], g["w"], P)
    p = np.random.default_rng(3).standard_normal(2 * N)
    np.testing.assert_allclose(A @ p, oracle.matvec(g["xs"], g["nrm"], g["w"], P, p), rtol=1e-12,
                               atol=1e-12 * np.max(np.abs(A @ p)))
    b = np.random.default_rng(4).standard_normal(2 * N)
    x_lu = np.linalg.solve(A, b)
    x, it, rr, ok = oracle.gmres(g["xs"], g["nrm"], g["w"], P, b, tol=1e-12, restart=60, maxit=2000)
    assert ok and rr < 1e-12
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-9


def test_born_exact_solution_residual_decreases():
    """Consistency: the discrete operator applied to the exact Born surface
    values (constant along normals) leaves a residual that falls under h-refinement."""
    R = 2.0
    res = []
    for h in (0.4, 0.2):
        g = oracle.sphere_nodes(R, h=h, eps=2 * h)
        N = g["w"].size
        P = oracle.Phys(1.0, 80.0, 0.1257, tau=h)
        ps, pn = cf.born_surface(R)
        p = np.concatenate([np.full(N, ps), np.full(N, pn)])
        b = oracle.rhs(g["xs"], g["nrm"], np.zeros((1, 3)), np.ones(1), 1.0)
        r = b - oracle.matvec(g["xs"], g["nrm"], g["w"], P, p)
        res.append(np.linalg.norm(r) / np.linalg.norm(b))
    assert res[1] < 0.7 * res[0]
    assert res[1] < 0.05


def test_born_solve_energy():
    """Born ion, R = 2, h = 0.25, band 3h: G_pol within a few percent of the
    closed form (Sec. 4.2), error below the tau = h case for tau = h/2."""
    R, h = 2.0, 0.25
    g = oracle.sphere_nodes(R, h=h, eps=3 * h)
    z, q = np.zeros((1, 3)), np.ones(1)
    b = oracle.rhs(g["xs"], g["nrm"], z, q, 1.0)
    Gs = cf.born_energy(R)
    errs = []
    for tau in (h, h / 2):
        P = oracle.Phys(1.0, 80.0, 0.1257, tau=tau)
        x, it, rr, ok = oracle.gmres(g["xs"], g["nrm"], g["w"], P, b, tol=1e-8)
        assert ok and it < 30
        G = oracle.gpol(q, oracle.psi_rxn(g["xs"], g["nrm"], g["w"], z, P, x))
        errs.append(abs(G - Gs) / abs(Gs))
    assert errs[0] < 0.05 and errs[1] < 0.03 and errs[1] < errs[0]
    assert Gs * oracle.KCAL_PER_E2_A == pytest.approx(-82.187, abs=2e-3)


@pytest.mark.slow
def test_table2_single_ion_64_half_tau():
    """Sec. 4.2 Table 2, 64^3, tau = h/2: solution and energy errors within 10%
    of the printed 5.93e-3 and 5.98e-3."""
    row = [r for r in _table2() if r[0] == 64 and r[1] == 0.5][0]
    n = 64
    h = 3.0 / n
    g = oracle.sphere_nodes(1.0, h=h, eps=2 * h)
    N = g["w"].size
    P = oracle.Phys(1.0, 80.0, 0.1257, tau=0.5 * h)
    z, q = np.zeros((1, 3)), np.ones(1)
    b = oracle.rhs(g["xs"], g["nrm"], z, q, 1.0)
    x, it, rr, ok = oracle.gmres(g["xs"], g["nrm"], g["w"], P, b, tol=1e-5)
    assert ok
    G = oracle.gpol(q, oracle.psi_rxn(g["xs"], g["nrm"], g["w"], z, P, x))
    Gs = cf.born_energy(1.0)
    ps, pn = cf.born_surface(1.0)
    w = g["w"]
    sol = np.sqrt((np.sum(w * (x[:N] - ps) ** 2) + np.sum(w * (x[N:] - pn) ** 2)) /
                  (np.sum(w) * (ps * ps + pn * pn)))
    assert abs(sol / row[4] - 1) < 0.1
    assert abs(abs(G - Gs) / abs(Gs) / row[6] - 1) < 0.1


# ---------------------------------------------------------------- Kirkwood series

def test_kirkwood_log_derivative_matches_scipy():
    x = 2.5
    ours = cf.kn_log_derivative(12, x)
    n = np.arange(13)
    ref = x * special.spherical_kn(n, x, derivative=True) / special.spherical_kn(n, x)
    np.testing.assert_allclose(ours, ref, rtol=1e-12)


def test_kirkwood_centre_charge_is_born():
    """n = 0 term only (charge at the centre): the series reduces to Born."""
    for kappa in (0.0, 0.1257):
        E = cf.kirkwood_energy(2.0, np.zeros((1, 3)), np.ones(1), 1.0, 80.0, kappa)
        assert E == pytest.approx(cf.born_energy(2.0, 1.0, 1.0, 80.0, kappa), rel=1e-13)


def test_kirkwood_kappa_zero_classical_coefficients():
    """kappa = 0: c_n = (n+1)(eps_I - eps_E)/(n eps_I + (n+1) eps_E)."""
    n = np.arange(30)
    ref = (n + 1) * (2.0 - 80.0) / (n * 2.0 + (n + 1) * 80.0)
    np.testing.assert_allclose(cf.kirkwood_coeffs(29, 20.0, 2.0, 80.0, 0.0), ref, rtol=1e-14)
    # small kappa approaches the kappa = 0 coefficients
    np.testing.assert_allclose(cf.kirkwood_coeffs(29, 20.0, 2.0, 80.0, 1e-7), ref, rtol=1e-5)


def test_kirkwood_surface_values_satisfy_flux_continuity():
    """Interior series vs an independent exterior evaluation: the interface
    conditions of Sec. 1 (continuity of psi and eps dpsi/dn) hold when the
    exterior field is built from the same Bessel coefficients."""
    a, kappa, eps_in, eps_out = 5.0, 0.3, 2.0, 80.0
    z = np.array([[1.0, 0.5, -0.3]])
    q = np.array([1.0])
    nmax = 60
    cn = cf.kirkwood_coeffs(nmax, a, eps_in, eps_out, kappa)
    s = np.linalg.norm(z[0])
    u = z[0] / s
    pts = np.array([[a, 0, 0], [0, a, 0], [0, 0, -a], [a / np.sqrt(3)] * 3])
    psi, psin = cf.kirkwood_surface(pts, a, z, q, eps_in, eps_out, kappa, nmax)
    # exterior: psi_out = sum_n C_n k_n(kappa r) P_n; C_n fixed by continuity at r = a
    n = np.arange(nmax + 1)
    x = kappa * a
    kn = special.spherical_kn(n, x)
    knp = special.spherical_kn(n, x, derivative=True)
    Bn = q[0] * s ** n / (4 * np.pi * eps_in * a ** (2 * n + 1)) * cn
    Cn = (q[0] * s ** n / (4 * np.pi * eps_in * a ** (n + 1)) + Bn * a ** n) / kn
    for i, p in enumerate(pts):
        cosg = p @ u / a
        P = np.array([special.eval_legendre(k, cosg) for k in n])
        psi_out = np.sum(Cn * kn * P)
        dpsi_out = np.sum(Cn * kappa * knp * P)
        assert psi[i] == pytest.approx(psi_out, rel=1e-10)
        assert eps_in * psin[i] == pytest.approx(eps_out * dpsi_out, rel=1e-8)


@pytest.mark.slow
def test_kirkwood_solve_energy():
    """Whole solve with several off-centre charges vs the Kirkwood series."""
    a, h = 6.0, 0.4
    rng = np.random.default_rng(11)
    u = rng.standard_normal((5, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    z = u * (4.0 * rng.random(5) ** (1 / 3))[:, None]
    q = np.array([1.0, -1.0, 1.0, 1.0, -1.0])
    eps_in, eps_out, kappa = 2.0, 80.0, 0.1257
    g = oracle.sphere_nodes(a, h=h, eps=2 * h)
    P = oracle.Phys(eps_in, eps_out, kappa, tau=h / 2)
    b = oracle.rhs(g["xs"], g["nrm"], z, q, eps_in)
    x, it, rr, ok = oracle.gmres(g["xs"], g["nrm"], g["w"], P, b, tol=1e-7)
    assert ok
    G = oracle.gpol(q, oracle.psi_rxn(g["xs"], g["nrm"], g["w"], z, P, x))
    Gs = cf.kirkwood_energy(a, z, q, eps_in, eps_out, kappa)
    assert abs(G - Gs) / abs(Gs) < 0.02, (G, Gs)
