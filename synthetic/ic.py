"""Closed-form, seeded initial conditions in the (v, omega_2, U_1, U_3) state.

The wall-normal velocity v = u_2 and the wall-normal vorticity omega_2 are
generated directly per Fourier mode, so u_1 and u_3 (recovered by each side
from continuity and the definition of omega_2) are divergence-free by
construction.  Shapes vanish where the boundary conditions require:
v = dv/dy = 0 and omega_2 = 0 at y = +-1.
"""
import math

import numpy as np

_MASK64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on a Python int."""
    x = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def uniform01(seed, kx, kz, field):
    """Counter-based uniform deviate in [0, 1) for one (seed, mode, field)."""
    ctr = ((seed & 0xFFFFFFFF) << 32) | ((kx & 0xFFF) << 20) | (((kz + 2048) & 0xFFF) << 8) | (field & 0xFF)
    return (splitmix64(splitmix64(ctr)) >> 11) * (1.0 / (1 << 53))


def wavenumbers(Lx, Lz, Nx, Nz):
    """k_1 for kx = 0..Nx/2-1, integer kz and k_3 in FFT order (Nyquist flagged)."""
    nxh = Nx // 2
    k1 = 2.0 * math.pi / Lx * np.arange(nxh)
    kzi = np.array([j if j < Nz // 2 else j - Nz for j in range(Nz)])
    k3 = 2.0 * math.pi / Lz * kzi
    nyq = np.zeros(Nz, dtype=bool)
    nyq[Nz // 2] = True
    return k1, kzi, k3, nyq


def bulk_velocity_loglaw(re_tau):
    """U_b+ from integrating the log law (kappa = 0.4, B = 5.5): 2.5 ln Re_tau + 3."""
    return 2.5 * math.log(re_tau) + 3.0


def reichardt_profile(y, re_tau, kappa=0.41):
    """Reichardt (1951) mean profile U+(y+), y+ = (1 - |y|) Re_tau."""
    yp = (1.0 - np.abs(np.asarray(y, dtype=np.float64))) * re_tau
    return (np.log1p(kappa * yp) / kappa
            + 7.8 * (1.0 - np.exp(-yp / 11.0) - (yp / 11.0) * np.exp(-yp / 3.0)))


def _trapz(f, y):
    return float(np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(y)))


def _uniform01_vec(seed, kx, kz, field):
    """uniform01 for an array of kx at one (seed, kz, field): the same integers in uint64."""
    m = np.uint64(_MASK64)
    kx = np.asarray(kx, dtype=np.uint64)
    ctr = (np.uint64((seed & 0xFFFFFFFF) << 32) | ((kx & np.uint64(0xFFF)) << np.uint64(20))
           | np.uint64((((kz + 2048) & 0xFFF) << 8) | (field & 0xFF)))

    def sm(x):
        with np.errstate(over="ignore"):
            x = (x + np.uint64(0x9E3779B97F4A7C15)) & m
            z = ((x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & m
            z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & m
        return z ^ (z >> np.uint64(31))

    return (sm(sm(ctr)) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def _fill(y, Lx, Lz, Nx, Nz, seed, mode_ok, amp_of_k):
    """Random-phase modes with shapes v ~ (1-y^2)^2 (1 + r y), omega_2 ~ k (1-y^2)(1 + s y).

    Returns unit-scaled (v, omega_2) and the volume-mean square of the
    perturbation velocity they imply, computed from analytic y-derivatives of
    the shapes and trapezoid weights in y.  ``mode_ok(kx, kz)`` and
    ``amp_of_k(k)`` take an array of kx (one kz at a time) and an array of |k|.
    The modes of one kz row are generated together; every value is the one a
    mode-by-mode loop would give.
    """
    y = np.asarray(y, dtype=np.float64)
    Ny = y.size
    nxh = Nx // 2
    k1, kzi, k3, nyq = wavenumbers(Lx, Lz, Nx, Nz)
    v = np.zeros((Ny, Nz, nxh), dtype=np.complex128)
    om = np.zeros_like(v)
    ms = np.zeros(Ny)
    w = (1.0 - y * y)[:, None]
    w2 = w * w
    yc = y[:, None]
    kxs = np.arange(nxh)
    for jz in range(Nz):
        kz = int(kzi[jz])
        if nyq[jz]:
            continue
        sel = np.asarray(mode_ok(kxs, kz), dtype=bool) & ~((kxs == 0) & (kz <= 0))
        kx = kxs[sel]
        if kx.size == 0:
            continue
        k2 = k1[kx] ** 2 + k3[jz] ** 2
        k = np.sqrt(k2)
        a = np.asarray(amp_of_k(k), dtype=np.float64) * np.ones_like(k)
        r = 2.0 * _uniform01_vec(seed, kx, kz, 2) - 1.0
        s_ = 2.0 * _uniform01_vec(seed, kx, kz, 3) - 1.0
        th = 2.0 * math.pi * _uniform01_vec(seed, kx, kz, 0)
        ph = 2.0 * math.pi * _uniform01_vec(seed, kx, kz, 1)
        ry = 1.0 + r * yc
        f = w2 * ry
        fp = -4.0 * yc * w * ry + w2 * r
        g = k * w * (1.0 + s_ * yc)
        vh = f * (a * np.exp(1j * th))
        oh = g * (a * np.exp(1j * ph))
        cols = slice(kx[0], kx[-1] + 1) if kx[-1] - kx[0] + 1 == kx.size else kx
        v[:, jz, cols] = vh
        om[:, jz, cols] = oh
        # |u_1|^2 + |u_3|^2 = (|dv/dy|^2 + |omega_2|^2) / k^2 for u_1 = i (k1 dv - k3 om) / k^2,
        # u_3 = i (k3 dv + k1 om) / k^2 (the cross terms cancel); a kx > 0 mode stands for
        # itself and its conjugate, a kx = 0 pair likewise
        a2 = a * a
        ms += 2.0 * ((f * f + (fp * fp + g * g) / k2) @ a2)
        if kx[0] == 0:   # kx = 0, kz > 0: its Hermitian partner at -kz
            jneg = (Nz - kz) % Nz
            v[:, jneg, 0] = np.conj(vh[:, 0])
            om[:, jneg, 0] = np.conj(oh[:, 0])
    return v, om, _trapz(ms, y) / 2.0


def perturbed_poiseuille(y, re_tau, Lx, Lz, Nx, Nz, seed, amp=0.1, kmax=4):
    """Laminar Poiseuille profile plus a divergence-free perturbation.

    U_1 = 1.5 U_b (1 - y^2) with U_b = 2.5 ln Re_tau + 3; perturbation in the
    modes |kx|, |kz| <= kmax with unit spectral amplitudes, scaled so that its
    rms velocity is ``amp * U_b``.  ``amp = 0`` gives the pure laminar state.
    """
    y = np.asarray(y, dtype=np.float64)
    ub = bulk_velocity_loglaw(re_tau)
    v, om, ms = _fill(y, Lx, Lz, Nx, Nz, seed, lambda kx, kz: (kx <= kmax) & (abs(kz) <= kmax),
                      lambda k: 1.0)
    scale = amp * ub / math.sqrt(ms) if ms > 0 else 0.0
    return dict(v=v * scale, omega2=om * scale, U1=1.5 * ub * (1.0 - y * y),
                U3=np.zeros_like(y), Ub=ub)


def turbulent_like(y, re_tau, Lx, Lz, Nx, Nz, seed, urms=1.0):
    """Reichardt mean profile plus random-phase fluctuations in every mode.

    The 2-D spectral amplitude falls as (k/k0)^(-4/3), i.e. a k^(-5/3) shell
    spectrum; the perturbation is scaled to rms velocity ``urms`` (wall units).
    """
    y = np.asarray(y, dtype=np.float64)
    k0 = 2.0 * math.pi / max(Lx, Lz)
    v, om, ms = _fill(y, Lx, Lz, Nx, Nz, seed, lambda kx, kz: np.ones(np.shape(kx), dtype=bool),
                      lambda k: (np.maximum(k, k0) / k0) ** (-4.0 / 3.0))
    scale = urms / math.sqrt(ms) if ms > 0 else 0.0
    return dict(v=v * scale, omega2=om * scale, U1=reichardt_profile(y, re_tau),
                U3=np.zeros_like(y), Ub=None)


def single_mode(y, Nx, Nz, kx, jz, v_profile=None, omega_profile=None, U1=None, U3=None):
    """State with one Fourier mode (and its Hermitian partner when kx = 0)."""
    y = np.asarray(y, dtype=np.float64)
    Ny = y.size
    v = np.zeros((Ny, Nz, Nx // 2), dtype=np.complex128)
    om = np.zeros_like(v)
    if v_profile is not None:
        v[:, jz, kx] = v_profile
    if omega_profile is not None:
        om[:, jz, kx] = omega_profile
    if kx == 0 and jz != 0:
        jneg = (Nz - jz) % Nz
        v[:, jneg, 0] = np.conj(v[:, jz, 0])
        om[:, jneg, 0] = np.conj(om[:, jz, 0])
    return dict(v=v, omega2=om,
                U1=np.zeros(Ny) if U1 is None else np.asarray(U1, dtype=np.float64),
                U3=np.zeros(Ny) if U3 is None else np.asarray(U3, dtype=np.float64))
