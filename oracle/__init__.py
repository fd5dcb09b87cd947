"""Plain, slow, obviously-correct FP64 CPU oracle for the RK4 time step of the
driven-dissipative Gross-Pitaevskii / dNLSE solver (PHOENIX, arXiv 2411.18341).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code, header, helper, table or constant with the CUDA path.

Modules
-------
``gp``     -- right-hand side of Eqs. (PULSE_psi)/(PULSE_res), the 5-point
              Laplacian of Sec. III.B.6, RK4 of Eqs. (rk4_K1)-(rk4_final),
              norm / energy / steady-state residual, stability limit.
``noise``  -- counter-based Philox4x32-10 (Salmon et al., SC'11) and a
              Box-Muller transform built only from correctly rounded FP32
              +, -, *, /, sqrt, so that the GPU can reproduce it bit for bit.
"""
from . import gp, noise  # noqa: F401
