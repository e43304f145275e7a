"""CPU oracle for the channel substep: TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of one semi-implicit low-storage RK3 substep
of the velocity-vorticity (v - omega_2) channel DNS of Vela-Martin et al.
(arXiv:1808.06461, Appendix A), with the sharp / box filter and the
filtered stresses tau_ij of Section 3.1.  Library primitives (numpy FFTs,
dense LAPACK solves, mpmath for the compact-scheme coefficient systems)
serve as steps; nothing is blocked, fused or reordered.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path and must
never be used as a fallback for it.

Parity: every function is pinned by the ``-m "not gpu"`` tests against
closed forms, invariants or brute force, except where its docstring says
"parity unpinned".
"""
from .channel import (RK3, ygrid, compact_coeffs, Setup, initial_state, substep, run,
                      velocities, to_physical, to_fourier, filter_transfer, filter_stresses,
                      stats, divergence, apply_y, nonlinear, rhs_terms, filtered_enstrophy, database_record,
                      retained_modes, spectra, helmholtz_error, pressure_solve,
                      filtered_pressure, SHARP, BOX, PAIRS)

__all__ = ["RK3", "ygrid", "compact_coeffs", "Setup", "initial_state", "substep", "run",
           "velocities", "to_physical", "to_fourier", "filter_transfer", "filter_stresses",
           "stats", "divergence", "apply_y", "nonlinear", "rhs_terms", "filtered_enstrophy", "database_record",
           "retained_modes", "spectra", "helmholtz_error", "pressure_solve",
           "filtered_pressure", "SHARP", "BOX", "PAIRS"]
