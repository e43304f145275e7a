"""Seeded synthetic inputs for the channel substep.

This module is shared by the tests, ``bench.py`` and ``__graft_entry__``: it
builds the initial states that both the CPU oracle and the CUDA path consume.
It holds none of the method's arithmetic: no compact finite differences, no
Fourier transforms, no time stepping.  The wall-normal grid is an argument
(each side builds its own); the profiles are evaluated from closed-form
shape functions, and the only derivatives taken are analytic derivatives of
those shape functions (used to set the perturbation amplitude).

Random numbers come from a counter-based generator (SplitMix64 of
(seed, kx, kz, field)), so a mode's phase does not depend on the order in
which modes are generated.

Field layout of every Fourier array returned here: complex128 of shape
(Ny, Nz, Nx // 2), index [j, jz, kx] with kx = 0 .. Nx/2-1 and jz in FFT
order (kz = jz for jz < Nz/2, kz = jz - Nz otherwise; jz = Nz/2 is the
Nyquist mode and is always zero).
"""
from .ic import (splitmix64, uniform01, bulk_velocity_loglaw, reichardt_profile,
                 perturbed_poiseuille, turbulent_like, single_mode, wavenumbers)
from .os_mode import orr_sommerfeld_mode, os_squire_mode

__all__ = ["splitmix64", "uniform01", "bulk_velocity_loglaw", "reichardt_profile",
           "perturbed_poiseuille", "turbulent_like", "single_mode", "wavenumbers",
           "orr_sommerfeld_mode", "os_squire_mode"]
