"""FP64 CPU oracle for the IBIM linearized Poisson-Boltzmann method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA library (its C source is ``ibim_oracle.c``,
compiled with gcc by ``oracle.build``).
"""
from .oracle import *  # noqa: F401,F403
from .closed_forms import *  # noqa: F401,F403
from . import warmstart_ref  # noqa: F401,E402
