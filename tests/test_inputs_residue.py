"""CPU checks of the protein-density input generator (inputs.residue_atoms):
seeded and repeatable, atoms no closer than the contact distance, net charge
zero, and a packing density well above the bead globule's."""
import numpy as np
import pytest

from paper_1709_08070_gb300 import inputs


def test_residue_atoms_is_seeded_and_respects_contacts():
    z1, r1, q1 = inputs.residue_atoms(400, seed=3)
    z2, r2, q2 = inputs.residue_atoms(400, seed=3)
    np.testing.assert_array_equal(z1, z2)
    np.testing.assert_array_equal(r1, r2)
    assert 300 <= len(z1) <= 400
    d = np.linalg.norm(z1[:, None, :] - z1[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 2.2 - 1e-12
    assert abs(q1.sum()) < 1e-12
    assert np.all((r1 >= 1.6) & (r1 <= 1.9))


def test_residue_atoms_pack_denser_than_the_bead_globule():
    """Atoms per convex-hull volume: about 1/21 per A^3 here (heavy atoms of a
    folded protein: about 1/17), against about 1/32 for the bead globule."""
    spatial = pytest.importorskip("scipy.spatial")
    z, r, q = inputs.residue_atoms(800, seed=4)
    zb, rb, qb = inputs.globule_atoms(len(z), seed=4)

    def atoms_per_volume(x):
        return len(x) / spatial.ConvexHull(x).volume

    assert atoms_per_volume(z) > 1.3 * atoms_per_volume(zb)
