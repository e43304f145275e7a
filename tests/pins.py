"""Measurements behind the oracle pins that more than one test module uses.

Each function runs the CPU oracle on a case whose answer the mathematics
fixes and returns how far the oracle is from it; the pin tests assert the
bound, and the planted-mistake tests assert that a mistake planted in the
oracle pushes the same measurement past it.  Oracle functions are looked up
through ``oracle.channel`` at call time, so a planted replacement is seen.
"""
import math

import numpy as np

import oracle.channel as OC
import synthetic as SY


def oblique_mode_rates(alpha=2.0, beta=1.0, re=7500.0, nsub=300, ny=97, dt=0.02):
    """Oblique Orr-Sommerfeld-Squire mode of plane Poiseuille flow through the substep.

    The box holds the single mode (k_1, k_3) = (alpha, beta) (Lx = 2 pi / alpha,
    Lz = 2 pi / beta) on U_1 = 1 - y^2 with nu = 1 / re, started from the
    coupled linear eigenmode (v, omega_2) at amplitude 1e-6.  Linear theory
    (Squire's transformation: c equals the two-dimensional eigenvalue at
    wavenumber k = sqrt(alpha^2 + beta^2) and Reynolds number re alpha / k)
    makes both |v| and |omega_2| change at the rate alpha c_i, and keeps
    omega_2 / v at the eigenmode's profile ratio.  omega_2 is driven by the
    Squire coupling -i beta U' v = i k_3 H_1 (linear part), advected by
    -i alpha U omega_2 = -i k_1 H_3 (linear part of H_3 = u_1 omega_2 - ...),
    and the omega_2 terms of H_1, H_2, H_3 must cancel in N_chi for v to
    follow the Orr-Sommerfeld rate.

    Returns (rate, rate_v, rate_omega2, profile_error): the linear-theory rate
    alpha c_i, the two measured amplitude rates, and the largest deviation of
    omega_2 / v(peak) from the eigenmode's ratio, relative to its maximum.
    """
    st = OC.Setup(re, 2 * math.pi / alpha, 2 * math.pi / beta, 4, ny, 4, dt, grid_re=180)
    c, vp, ep = SY.os_squire_mode(re, alpha, beta, st.y)
    S0 = SY.single_mode(st.y, 4, 4, 1, 1, v_profile=1e-6 * vp, omega_profile=1e-6 * ep,
                        U1=1.0 - st.y ** 2)
    S = OC.initial_state(st, S0["v"], S0["omega2"], S0["U1"], S0["U3"])

    def amp(F):
        return math.sqrt(np.sum(st.wq * np.abs(F[:, 1, 1]) ** 2))

    av, aw, t0 = amp(S["v"]), amp(S["omega2"]), S["t"]
    S = OC.run(st, S, nsub)
    T = S["t"] - t0
    rv = math.log(amp(S["v"]) / av) / T
    rw = math.log(amp(S["omega2"]) / aw) / T
    j = int(np.argmax(np.abs(vp)))
    ratio = S["omega2"][:, 1, 1] / S["v"][j, 1, 1]
    prof = float(np.abs(ratio - ep / vp[j]).max() / np.abs(ep / vp[j]).max())
    return alpha * c.imag, rv, rw, prof


def energy_residual(st, S):
    """Largest |sum_k w Re(conj(u_k) . H_k)| over heights, relative to sum_k w |u_k| |H_k|.

    H = P(u x omega) from ``nonlinear``; u holds only retained modes, and the
    3/2 rule makes P(u x omega) exact on them, so the Parseval sum equals the
    plane mean of u . (u x omega), which vanishes identically: the sum is zero
    to rounding at every height, whatever the flow.
    """
    H = OC.nonlinear(st, S)
    u1, v, u3, _, _, _ = OC.velocities(st, S)
    w = np.where(np.arange(st.nxh) == 0, 1.0, 2.0)[None, None, :]
    dot = sum(np.sum(w * (np.conj(a) * b).real, axis=(1, 2)) for a, b in zip((u1, v, u3), H))
    mag = sum(np.sum(w * np.abs(a) * np.abs(b), axis=(1, 2)) for a, b in zip((u1, v, u3), H))
    return float(np.max(np.abs(dot)) / np.max(mag))


def vorticity_divergence(st, S):
    """max |i k_1 omega_1 + D1 omega_2 + i k_3 omega_3| relative to max |D1 omega_2|.

    The divergence of a curl vanishes; with the velocities of ``velocities``
    (omega_2 = i k_3 u_1 - i k_1 u_3 by construction) the identity holds for
    the discrete D1 too, since D1 acts on each mode linearly.
    """
    u1, v, u3, du1, dv, du3 = OC.velocities(st, S)
    om1, om2, om3 = OC.vorticity(st, S, u1, v, u3, du1, du3)
    d2 = OC.apply_y(st.D1, om2)
    div = 1j * st.K1 * om1 + d2 + 1j * st.K3 * om3
    return float(np.abs(div).max() / np.abs(d2).max())
