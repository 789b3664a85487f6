"""Failure path of the bounded device waits, exercised without a GPU fault.

A kernel whose bounded wait gives up records IBIM_ERR_DEVICE_TIMEOUT in its
context's device error word and returns; the host reads the word at the next
synchronising call.  Here the bit is set from the host side of an ordinary,
complete launch (ibim_debug_raise_device_error), no wait is made to give up:
the synchronising call must report the status, and the very next call on the
same context must succeed and agree with the FP64 oracle.
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

TIMEOUT = 6  # IBIM_ERR_DEVICE_TIMEOUT


def _worst(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_timeout_status_is_reported_and_the_context_recovers():
    xs, nr, w = inputs.sphere_cloud(700, radius=4.0, seed=12)
    N = xs.shape[0]
    ctx = ibim.Context.from_nodes(xs, nr, w, h=0.3)
    try:
        P = ibim.Phys(2.0, 80.0, 0.1257, 0.3, 0)
        Po = oracle.Phys(2.0, 80.0, 0.1257, 0.3, 0)
        p = inputs.random_vector(2 * N, seed=13)
        yo = oracle.matvec(xs, nr, w, Po, p)
        for prec, tol in ((ibim.IBIM_F32C, 1e-5), (ibim.IBIM_F64, 1e-10)):
            ibim.ibim_debug_raise_device_error(ctx.handle, TIMEOUT)
            with pytest.raises(ibim.IbimError) as e:
                ctx.matvec_host(P, p, precision=prec)
            assert e.value.status == TIMEOUT and "gave up" in str(e.value)
            y = ctx.matvec_host(P, p, precision=prec)  # the word was cleared: the next call succeeds
            for blk in (slice(0, N), slice(N, 2 * N)):
                assert _worst(y[blk], yo[blk]) < tol, prec
        # a solve reads the word at its end as well, and the next solve succeeds
        ctx.set_charges(np.array([[0.3, -0.2, 0.1]]), np.array([1.0]))
        dp = torch.empty(2 * N, dtype=torch.float64, device="cuda")
        ibim.ibim_debug_raise_device_error(ctx.handle, TIMEOUT)
        with pytest.raises(ibim.IbimError) as e:
            ctx.solve(P, dp, precision=ibim.IBIM_F32C, tol=1e-8, restart=64, maxit=200)
        assert e.value.status == TIMEOUT
        info = ctx.solve(P, dp, precision=ibim.IBIM_F32C, tol=1e-8, restart=64, maxit=200)
        assert info["converged"]
        b = oracle.rhs(xs, nr, np.array([[0.3, -0.2, 0.1]]), np.array([1.0]), 2.0)
        r = b - oracle.matvec(xs, nr, w, Po, dp.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-6
        with pytest.raises(ibim.IbimError) as e:
            ibim.ibim_debug_raise_device_error(ctx.handle, 4)  # only the timeout status can be raised
        assert e.value.status == 1
    finally:
        ctx.close()
