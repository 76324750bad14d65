"""FP64 CPU oracle for the ADMM iteration (Zhou & Bhattacharya, Section 2).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct numpy code that the
CUDA path is compared against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library and never imports the solver package.
"""
from .admm import (admm_solve, u_step, grad_u, grad_from_spectrum, local_newton, wavenumbers,
                   rms, initial_state, homogenised_stress, local_newton_lce, frank_force,
                   tangent_basis, retract)
from .materials import NeoHookean, LinearElastic, LCE, make_material, make_lce
