"""Closed-form solutions used to pin the oracle (test infrastructure only).

* Born ion (Sec. 4.2, the single-ion model): potential, surface values and
  polarization energy of one charge at the centre of a sphere.
* Kirkwood series for point charges inside a dielectric sphere in a
  screening exterior, written out from the linearized PB equation of Sec. 1
  (separation of variables; interior Legendre series, exterior modified
  spherical Bessel functions of the second kind).  Energies are in e^2/A with
  the paper's psi = q/(4 pi eps r) convention.
"""
import numpy as np

__all__ = ["born_energy", "born_surface", "born_potential", "kirkwood_coeffs",
           "kirkwood_psi_rxn", "kirkwood_energy", "kirkwood_surface", "kn_log_derivative"]


def born_energy(R, q=1.0, eps_in=1.0, eps_out=80.0, kappa=0.1257):
    """G*_pol = q^2/(8 pi R) (1/(eps_E (1 + kappa R)) - 1/eps_I) (Sec. 4.2)."""
    return q * q / (8.0 * np.pi * R) * (1.0 / (eps_out * (1.0 + kappa * R)) - 1.0 / eps_in)


def born_potential(x, R, q=1.0, eps_in=1.0, eps_out=80.0, kappa=0.1257):
    """psi*(x) of Sec. 4.2 (exterior uses eps = eps_E, continuity at |x| = R)."""
    r = np.linalg.norm(np.atleast_2d(x), axis=1)
    inside = q / (4 * np.pi * eps_in * r) + q / (4 * np.pi * R) * (1 / (eps_out * (1 + kappa * R)) - 1 / eps_in)
    outside = q * np.exp(-kappa * (r - R)) / (4 * np.pi * eps_out * (1 + kappa * R) * r)
    return np.where(r < R, inside, outside)


def born_surface(R, q=1.0, eps_in=1.0, eps_out=80.0, kappa=0.1257):
    """(psi, psi_n) on the sphere; psi_n is the interior-side normal derivative."""
    psi = q / (4 * np.pi * eps_out * (1 + kappa * R) * R)
    psin = -q / (4 * np.pi * eps_in * R * R)
    return psi, psin


def kn_log_derivative(nmax, x):
    """x k_n'(x)/k_n(x) for n = 0..nmax, k_n the modified spherical Bessel
    function of the second kind, through the ratio R_n = k_{n+1}/k_n:
    R_0 = 1 + 1/x, R_n = 1/R_{n-1} + (2n+1)/x (upward, stable for k_n),
    and x k_n'/k_n = n - x R_n."""
    out = np.empty(nmax + 1)
    Rn = 1.0 + 1.0 / x
    for n in range(nmax + 1):
        if n > 0:
            Rn = 1.0 / Rn + (2 * n + 1) / x
        out[n] = n - x * Rn
    return out


def kirkwood_coeffs(nmax, a, eps_in, eps_out, kappa):
    """c_n = (gamma_n + (n+1) eps_I) / (n eps_I - gamma_n), gamma_n = eps_E x k_n'/k_n
    at x = kappa a; for kappa = 0, gamma_n = -(n+1) eps_E."""
    n = np.arange(nmax + 1, dtype=np.float64)
    if kappa == 0.0:
        gam = -(n + 1.0) * eps_out
    else:
        gam = eps_out * kn_log_derivative(nmax, kappa * a)
    return (gam + (n + 1.0) * eps_in) / (n * eps_in - gam)


def _legendre_all(nmax, t):
    """P_0..P_nmax at the points t (Bonnet recurrence); shape (nmax+1, len(t))."""
    t = np.asarray(t, dtype=np.float64)
    P = np.empty((nmax + 1,) + t.shape)
    P[0] = 1.0
    if nmax >= 1:
        P[1] = t
    for n in range(1, nmax):
        P[n + 1] = ((2 * n + 1) * t * P[n] - n * P[n - 1]) / (n + 1)
    return P


def kirkwood_psi_rxn(points, a, z, q, eps_in, eps_out, kappa, nmax=200, centre=(0.0, 0.0, 0.0)):
    """Reaction potential at interior points:
    psi_rxn(x) = sum_k q_k/(4 pi eps_I) sum_n c_n (r s_k)^n / a^(2n+1) P_n(cos gamma_k)."""
    c0 = np.asarray(centre, dtype=np.float64)
    X = np.atleast_2d(np.asarray(points, dtype=np.float64)) - c0
    Z = np.atleast_2d(np.asarray(z, dtype=np.float64)) - c0
    q = np.asarray(q, dtype=np.float64)
    cn = kirkwood_coeffs(nmax, a, eps_in, eps_out, kappa)
    r = np.linalg.norm(X, axis=1)
    s = np.linalg.norm(Z, axis=1)
    out = np.zeros(X.shape[0])
    for k in range(Z.shape[0]):
        denom = np.maximum(r * s[k], 1e-300)
        cosg = np.where(r * s[k] > 0, (X @ Z[k]) / denom, 1.0)
        cosg = np.clip(cosg, -1.0, 1.0)
        P = _legendre_all(nmax, cosg)
        n = np.arange(nmax + 1)[:, None]
        ratio = (r * s[k] / (a * a))[None, :] ** n
        out += q[k] / (4 * np.pi * eps_in) * np.sum(cn[:, None] * ratio * P, axis=0) / a
    return out


def kirkwood_energy(a, z, q, eps_in, eps_out, kappa, nmax=200, centre=(0.0, 0.0, 0.0)):
    """G_pol = 1/2 sum_j q_j psi_rxn(z_j) (e^2/A)."""
    psi = kirkwood_psi_rxn(z, a, z, q, eps_in, eps_out, kappa, nmax, centre)
    return 0.5 * float(np.dot(np.asarray(q, dtype=np.float64), psi))


def kirkwood_surface(points, a, z, q, eps_in, eps_out, kappa, nmax=200, centre=(0.0, 0.0, 0.0)):
    """(psi, psi_n) at surface points |x - centre| = a from the interior series:
    psi = sum_k q_k/(4 pi eps_I |x - z_k|) + psi_rxn, psi_n the interior-side radial
    derivative (Coulomb part differentiated in closed form, series termwise)."""
    c0 = np.asarray(centre, dtype=np.float64)
    X = np.atleast_2d(np.asarray(points, dtype=np.float64)) - c0
    Z = np.atleast_2d(np.asarray(z, dtype=np.float64)) - c0
    q = np.asarray(q, dtype=np.float64)
    cn = kirkwood_coeffs(nmax, a, eps_in, eps_out, kappa)
    r = np.linalg.norm(X, axis=1)
    nrm = X / r[:, None]
    s = np.linalg.norm(Z, axis=1)
    psi = np.zeros(X.shape[0])
    psin = np.zeros(X.shape[0])
    n = np.arange(nmax + 1)[:, None]
    for k in range(Z.shape[0]):
        d = X - Z[k]
        dist = np.linalg.norm(d, axis=1)
        psi += q[k] / (4 * np.pi * eps_in * dist)
        psin += -q[k] * np.sum(d * nrm, axis=1) / (4 * np.pi * eps_in * dist ** 3)
        cosg = np.clip((X @ Z[k]) / np.maximum(r * s[k], 1e-300), -1.0, 1.0)
        P = _legendre_all(nmax, cosg)
        t = (r * s[k] / (a * a))[None, :] ** n  # (r s)^n / a^(2n)
        term = cn[:, None] * t * P / a  # c_n (r s)^n / a^(2n+1) P_n
        psi += q[k] / (4 * np.pi * eps_in) * np.sum(term, axis=0)
        # d/dr of r^n: n r^(n-1) = n r^n / r
        psin += q[k] / (4 * np.pi * eps_in) * np.sum(term * n, axis=0) / r
    return psi, psin
