"""Plain FP64 CPU oracle for the generalized Poisson / Poisson-Boltzmann PCG.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library; the only
common module is ``synth`` (seeded inputs, no solver arithmetic).

Every function follows a passage of arXiv:1509.00680 (cited by section,
equation or algorithm) or a stated reading of it.  NumPy/SciPy FP64 only; a
library FFT or dense solve serves as a step, with no fusion or reordering.

Modules
  constants  physical constants and the electrolyte conversions (Eq. rhoions)
  fd16       order-16 central finite differences (Sec. "Numerical results")
  green      vacuum Poisson solve S for free/periodic/surface BC (Eq. SPe)
  operators  s = eps^-1/2, q = sqrt(eps) lap sqrt(eps), M = s S(s .)  (Eq. PCGdef, corr)
  pcg        Algorithm 2 (PCG) for the GPe and linear PB (Eq. corr, corrPB)
  pb         ionic charge (Eq. rhoions, ionsconcPB) and Algorithms 3 and 4
  dense      dense assembly of the discrete operator, direct and Newton solves
  sc         Algorithm 1 (SC) and PSD / PSD+DIIS comparison solvers (Eqs. remap, rhoiter, PrePSD)
  dft        sccs dielectric, polarization charge, v_eps, electrostatic energy (Eqs. sccs, rhopol, veps)
"""
from . import constants, fd16, green, operators, pcg, pb, dense, sc, dft  # noqa: F401
from .pcg import solve_gpe, solve_lpb  # noqa: F401
from .pb import solve_nlpb  # noqa: F401
