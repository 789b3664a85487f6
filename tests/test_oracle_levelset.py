"""Pins of the oracle's level-set construction (Sec. 3.1-3.2) against geometry
whose solvent excluded surface is known in closed form.

* One atom: the SES is the atom's sphere, so phi must be |x - z| - r in the band
  and the band nodes/area must agree with the analytic-sphere band.
* Two atoms closer than 2 (r + rho0): in the mid-plane the SES is the inner
  rim of the torus swept by the probe, at radius a - rho0 with
  a = sqrt((r + rho0)^2 - (d/2)^2); there phi = s - (a - rho0).
* A closed shell of atoms: the inner surface bounds a cavity that the
  cavity removal of Sec. 3.1.2 must delete.
"""
import numpy as np
import pytest

import oracle


def test_single_atom_phi_is_distance_to_sphere():
    r, h = 2.0, 0.25
    eps = 2 * h
    st = oracle.ls_steps(np.zeros((1, 3)), np.array([r]), probe=1.4, h=h, eps=eps)
    X = oracle.grid_coords(st["grid"])
    d = np.linalg.norm(X, axis=-1) - r
    band = np.abs(d) < eps
    assert np.max(np.abs(st["sas"][band] - (d[band] - 1.4))) < 1e-12  # phi_SAS = F - rho0
    assert np.max(np.abs(st["flowed"][band] - d[band])) < 2e-4
    assert np.max(np.abs(st["phi"][band] - d[band])) < 2e-4
    assert st["changed"] == 0  # no cavity
    b = oracle.ls_band(st["grid"], st["phi"], eps)
    s = oracle.sphere_nodes(r, h=h, eps=eps)
    assert abs(b["w"].size - s["w"].size) < 0.02 * s["w"].size
    assert abs(b["w"].sum() / s["w"].sum() - 1) < 1e-4
    # projections land on the sphere, normals are radial
    assert np.max(np.abs(np.linalg.norm(b["xs"], axis=1) - r)) < 1e-3
    cosang = np.sum(b["nrm"] * b["xs"], axis=1) / np.linalg.norm(b["xs"], axis=1)
    assert np.min(cosang) > 1 - 1e-5


def _neck_error(h):
    d0, rr, rho = 4.5, 1.8, 1.4
    eps = 2 * h
    z = np.array([[-d0 / 2, 0, 0], [d0 / 2, 0, 0]])
    st = oracle.ls_steps(z, np.array([rr, rr]), probe=rho, h=h, eps=eps)
    X = oracle.grid_coords(st["grid"])
    a = np.sqrt((rr + rho) ** 2 - (d0 / 2) ** 2)
    s = np.hypot(X[..., 1], X[..., 2])
    sel = (np.abs(X[..., 0]) < 1e-9) & (np.abs(s - (a - rho)) < eps)
    assert sel.sum() > 20
    return np.max(np.abs(st["phi"][sel] - (s[sel] - (a - rho))))


def test_two_atom_neck_is_torus_rim():
    """The neck radius a - rho0 = 0.875 A is under two cells at h = 0.5 (coarser than
    the paper's h ~ min(rho0, r, 2 eps)/7 guidance) and well resolved at h = 0.25."""
    e_coarse, e_fine = _neck_error(0.5), _neck_error(0.25)
    assert e_coarse < 0.1 and e_fine < 0.008
    assert e_fine < e_coarse / 8  # better than third order between the two grids


def _shell(n=300, Rs=9.0):
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = np.pi * (1 + 5 ** 0.5) * i
    return Rs * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)


def test_cavity_inside_closed_shell_is_removed():
    z = _shell()
    r = np.full(len(z), 1.8)
    h, eps = 0.5, 1.0
    st = oracle.ls_steps(z, r, probe=1.4, h=h, eps=eps)
    X = oracle.grid_coords(st["grid"])
    rad = np.linalg.norm(X, axis=-1)
    # before removal the flowed level set has an inner surface (phi > 0 inside the shell)
    assert np.any((st["flowed"] > 0) & (rad < 6.0))
    assert np.any(st["labels"] == 2)
    assert np.all(st["labels"][rad < 5.0] != 1)  # the void is not reachable from outside
    assert st["changed"] > 0
    b = oracle.ls_band(st["grid"], st["phi"], eps)
    br = np.linalg.norm(b["xs"], axis=1)
    assert b["w"].size > 0
    assert np.min(br) > 9.0  # only the outer surface remains in the band
