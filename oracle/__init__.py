"""FP64 CPU oracle for the Roman-Perez--Soler evaluation of E_c^nl and v_nl.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (its own quadrature, splines, radial transform, FFT driver,
energy and potential), so agreement between the two is evidence, not
tautology.

Modules
-------
vdw_oracle   plain numpy FP64 statement of every step, in the paper's order.
dion.c       the Dion kernel phi(d1, d2) by direct double quadrature (compiled
             on first use with gcc into ``oracle/_build``).
learned      the learned reduced basis (a network's channel weights and a
             learned pair kernel in place of the splines), its potential,
             parameter gradients and training loss.
semilocal    the semilocal partner terms of Eq. (Exc): revPBE exchange and
             LDA correlation, and the total E_xc with its potential.
"""
from .vdw_oracle import *  # noqa: F401,F403
