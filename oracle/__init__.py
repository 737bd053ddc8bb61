"""FP64 CPU oracle for the gray-RTE source iteration and GSIS (steady and time-dependent).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import or run anything here.  The oracle shares no code
with the CUDA library and neither imports the other.

Parity pins (see tests/test_oracle_pins.py): every function here is checked
against closed forms, invariants or brute force on tiny inputs; none is
"parity unpinned".  The adjoint (oracle/adjoint.py) is pinned by
tests/test_oracle_adjoint.py: dot-product identities of each transposed step
against the forward oracle and central differences of full forward solves.
The time-dependent radiation-material steps (oracle/timedep.py) are pinned
by tests/test_oracle_timedep.py: brute-force solves of the fully implicit
and the Fleck-Cummings systems on tiny meshes, equilibrium preservation,
energy conservation and the long-step radiative-equilibrium limit.
The adjoint of a time-dependent GSIS run (oracle/td_adjoint.py) is pinned by
tests/test_oracle_td_adjoint.py: central differences of full forward runs
with respect to the opacities and the initial state.
The UW2 kinetic step (oracle/uw2.py) is pinned by tests/test_oracle_uw2.py:
exactness on linear fields, the Barth-Jespersen bound, the zero-limiter
reduction to the UW1 oracle, conservation, second-order convergence on a
manufactured solution and convergence in the diffusion limit.
"""
from .gsis import (  # noqa: F401
    angular_source, transport_sweep, alsm_gradient, high_order_terms, geometry, pseudo_time_shift,
    face_lists, gamma_coefficient, boundary_beta, synthetic_matrix, synthetic_rhs,
    SyntheticSolver, err_w, si_solve, gsis_solve, gsis_iteration, si_iteration,
)
