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


def _rows_every_variant(ctx, bo, inv, rows, h, seed, variants, with_f64=True):
    """Oracle rows `rows` (oracle numbering) of the operator on the shared node
    set against the library's, element by element per output block, for the
    FP64 path and the float-float path (1e-10) and each FP32 variant in
    `variants` at its occupancy-limited grid (1e-5)."""
    N = ctx.N
    P = ibim.Phys(1.0, 80.0, 0.1257, h, 0)
    Po = oracle.Phys(1.0, 80.0, 0.1257, h, 0)
    p_orc = inputs.random_vector(2 * N, seed=seed)
    p_gpu = np.empty(2 * N)
    p_gpu[inv] = p_orc[:N]
    p_gpu[N + inv] = p_orc[N:]
    y1o, y2o = oracle.matvec_rows(bo["xs"], bo["nrm"], bo["w"], Po, p_orc, rows)
    din = torch.from_numpy(p_gpu).cuda()
    dout = torch.empty_like(din)
    configs = ([(ibim.IBIM_F64, None, 1e-10)] if with_f64 else []) + [(ibim.IBIM_FF, None, 1e-10)] + \
        [(ibim.IBIM_F32C, v, 1e-5) for v in variants]
    for prec, v, tol in configs:
        if v is not None:
            ctx.set_f32_variant(v, 0)
        ctx.matvec(P, din, dout, precision=prec)
        y = dout.cpu().numpy()
        errs = []
        for got, ref in ((y[:N][inv[rows]], y1o), (y[N:][inv[rows]], y2o)):
            errs += [np.linalg.norm(got - ref) / np.linalg.norm(ref), np.max(np.abs(got - ref)) / np.max(np.abs(ref))]
        print("globule N=%d prec=%d variant %s: block 1 rel %.2e worst %.2e | block 2 rel %.2e worst %.2e"
              % (N, prec, v, *errs))
        assert max(errs) < tol, (prec, v, errs)


def test_globule_operator_on_gpu_geometry():
    """2,000-atom seeded globule, probe 1.4, h = 0.5, eps = 2h: geometry parity,
    then 2,048 operator rows on the shared nodes, element by element, for the
    FP64 path (1e-10) and every FP32 variant (1e-5)."""
    z, r, q = inputs.globule_atoms(2000)
    h = 0.5
    ctx, bo, bg, jg, jo = _compare(z, r, 1.4, h, 2 * h)
    N = ctx.N
    assert N > 50000
    assert len(jg) == N == len(bo["w"])  # identical node sets on this input
    inv = np.empty(N, dtype=np.int64)
    inv[jo] = jg  # oracle node -> gpu node
    rows = inputs.random_rows(N, 2048, seed=42)  # oracle rows
    _rows_every_variant(ctx, bo, inv, rows, h, 41, range(len(ibim.ibim_f32_variants())))
    ctx.close()


def test_ten_thousand_atom_globule_operator_rows():
    """A 10,000-atom globule of the learned-start evaluation size (about 740k
    nodes): geometry parity with the oracle's level set, then 1,024 seeded
    oracle rows of the FP32 operator (the autotuner's choice and both
    symmetric variants; 1e-5) and of the float-float operator (1e-10), element
    by element.  The plain FP64 operator is left out at this size (about a
    minute per application)."""
    z, r, q = inputs.globule_atoms(10000, seed=inputs.SEED_LEARNED + 10000)
    h = 0.5
    ctx, bo, bg, jg, jo = _compare(z, r, 1.4, h, 2 * h)
    N = ctx.N
    assert N > 500000
    assert len(jg) == N == len(bo["w"])
    inv = np.empty(N, dtype=np.int64)
    inv[jo] = jg
    P = ibim.Phys(1.0, 80.0, 0.1257, h, 0)
    tuned, _, _ = ctx.autotune(P)
    sym = [v for v, info in enumerate(ibim.ibim_f32_variants()) if info[3]]
    rows = inputs.random_rows(N, 1024, seed=43)
    _rows_every_variant(ctx, bo, inv, rows, h, 44, [tuned] + [v for v in sym if v != tuned], with_f64=False)
    ctx.close()
