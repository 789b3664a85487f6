"""GPU level-set SES construction (ibim_build) against the oracle's.

Both sides build the level set from the same atoms on the same grid.  The
final phi grids must agree to round-off, the band node sets must be equal
(apart from nodes whose |phi| sits within round-off of eps, whose weight is
zero), and the nodes' projections, normals and weights must agree.  On the
2,000-atom globule the FP32 and FP64 operators are then checked against the
oracle's operator on sampled rows of the shared node set.
"""
import numpy as np
import pytest

import oracle
from paper_1709_08070_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1709_08070_gb300 import ibim  # noqa: E402


def _shell(n=300, Rs=9.0):
    i = np.arange(n) + 0.5
    ph = np.arccos(1 - 2 * i / n)
    th = np.pi * (1 + 5 ** 0.5) * i
    return Rs * np.stack([np.cos(th) * np.sin(ph), np.sin(th) * np.sin(ph), np.cos(ph)], axis=1)


def _compare(z, r, probe, h, eps, phi_tol=1e-9):
    ctx = ibim.Context.molecule(z, r, None, probe=probe, h=h, band_eps=eps)
    g, phi_o, changed = oracle.ls_ses(z, r, probe, h, eps)
    lo, n, phi_g = ctx.levelset()
    assert list(lo) == list(g.lo) and list(n) == list(g.n)
    dphi = np.max(np.abs(phi_g - phi_o))
    assert dphi < phi_tol, dphi
    bo = oracle.ls_band(g, phi_o, eps)
    bg = ctx.nodes()
    ko = {tuple(v): i for i, v in enumerate(bo["ijk"])}
    common = [(j, ko[tuple(v)]) for j, v in enumerate(bg["ijk"]) if tuple(v) in ko]
    only_g = [j for j, v in enumerate(bg["ijk"]) if tuple(v) not in ko]
    only_o = set(range(len(bo["w"]))) - {i for _, i in common}
    for j in only_g:
        assert abs(abs(bg["d"][j]) - eps) < 10 * phi_tol
    for i in only_o:
        assert abs(abs(bo["d"][i]) - eps) < 10 * phi_tol
    jg = np.array([a for a, _ in common])
    jo = np.array([b for _, b in common])
    np.testing.assert_allclose(bg["xs"][jg], bo["xs"][jo], rtol=0, atol=1e-8)
    np.testing.assert_allclose(bg["nrm"][jg], bo["nrm"][jo], rtol=0, atol=1e-8)
    np.testing.assert_allclose(bg["w"][jg], bo["w"][jo], rtol=0, atol=1e-9 * h ** 3)
    return ctx, bo, bg, jg, jo


def test_single_atom_levelset_matches_oracle():
    ctx, *_ = _compare(np.zeros((1, 3)), np.array([2.0]), 1.4, 0.25, 0.5)
    ctx.close()


def test_two_atom_neck_matches_oracle():
    z = np.array([[-2.25, 0, 0], [2.25, 0, 0]])
    ctx, *_ = _compare(z, np.array([1.8, 1.8]), 1.4, 0.25, 0.5)
    ctx.close()


def test_cavity_shell_matches_oracle():
    z = _shell()
    ctx, bo, bg, jg, jo = _compare(z, np.full(len(z), 1.8), 1.4, 0.5, 1.0)
    assert np.min(np.linalg.norm(bg["xs"], axis=1)) > 9.0
    ctx.close()


def test_globule_operator_on_gpu_geometry():
    """2,000-atom seeded globule, probe 1.4, h = 0.5, eps = 2h: geometry parity,
    then operator rows on the shared nodes (FP64 1e-10, FP32 1e-5)."""
    z, r, q = inputs.globule_atoms(2000)
    h = 0.5
    ctx, bo, bg, jg, jo = _compare(z, r, 1.4, h, 2 * h)
    N = ctx.N
    assert N > 50000
    assert len(jg) == N == len(bo["w"])  # identical node sets on this input
    P = ibim.Phys(1.0, 80.0, 0.1257, h, 0)
    Po = oracle.Phys(1.0, 80.0, 0.1257, h, 0)
    inv = np.empty(N, dtype=np.int64)
    inv[jo] = jg  # oracle node -> gpu node
    p_orc = inputs.random_vector(2 * N, seed=41)
    p_gpu = np.empty(2 * N)
    p_gpu[inv] = p_orc[:N]
    p_gpu[N + inv] = p_orc[N:]
    rows = inputs.random_rows(N, 1024, seed=42)  # oracle rows
    y1o, y2o = oracle.matvec_rows(bo["xs"], bo["nrm"], bo["w"], Po, p_orc, rows)
    din = torch.from_numpy(p_gpu).cuda()
    dout = torch.empty_like(din)
    for prec, tol in ((ibim.IBIM_F64, 1e-10), (ibim.IBIM_F32C, 1e-5)):
        ctx.matvec(P, din, dout, precision=prec)
        y = dout.cpu().numpy()
        e1 = np.linalg.norm(y[:N][inv[rows]] - y1o) / np.linalg.norm(y1o)
        e2 = np.linalg.norm(y[N:][inv[rows]] - y2o) / np.linalg.norm(y2o)
        print("globule N=%d prec=%d rel err %.3e %.3e" % (N, prec, e1, e2))
        assert max(e1, e2) < tol, (prec, e1, e2)
    ctx.close()
