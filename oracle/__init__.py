"""FP64 CPU oracle for the PNOF energy / orbital-Lagrangian build.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import it.  The CUDA library never does, and the
oracle never imports the CUDA library.

Pins (tests/test_oracle_pins.py) tie every function to something other than
itself: brute-force 4-index ERIs, the Roothaan Hartree-Fock limit, the APSG
determinant-space energy, the 2RDM contraction of Eqs. intra/interaa/interab,
the half-occupancy coincidence of PNOF7 and PNOF7s, central finite differences
and the Euler identity E = sum_p (lambda_pp + n_p H_pp).
"""
from . import pnof  # noqa: F401
