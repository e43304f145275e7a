"""Planted mistakes: each pin of the non-linear coupling catches a plausible slip.

A copy of one oracle function with one slip (a flipped sign, swapped
wavenumbers, a mis-signed vorticity term) replaces the original inside
``oracle.channel`` for one test, on the CPU; the test asserts that the pin
measuring that part of the method moves past the bound its pin test uses.
Together with the unmodified pins in ``test_oracle_pins.py`` this shows the
pins are sensitive to the parts of Appendix A's Eq. (hghv) and of
H = u x omega that the two-dimensional checks never exercise.
"""
import math

import numpy as np
import pytest

import oracle.channel as OC
import pins
import synthetic as SY


def _products(st, S):
    u1, v, u3, du1, dv, du3 = OC.velocities(st, S)
    om1, om2, om3 = OC.vorticity(st, S, u1, v, u3, du1, du3)
    p = [OC.to_physical(st, F) for F in (u1, v, u3, om1, om2, om3)]
    return p[:3], p[3:]


def _nonlinear_h3_flipped(st, S):
    u, w = _products(st, S)
    H1 = u[1] * w[2] - u[2] * w[1]
    H2 = u[2] * w[0] - u[0] * w[2]
    H3 = -u[0] * w[1] - u[1] * w[0]          # slip: sign of u_1 omega_2
    return tuple(OC.to_fourier(st, H) for H in (H1, H2, H3))


def _nonlinear_h1_flipped(st, S):
    u, w = _products(st, S)
    H1 = u[1] * w[2] + u[2] * w[1]           # slip: sign of u_3 omega_2
    H2 = u[2] * w[0] - u[0] * w[2]
    H3 = u[0] * w[1] - u[1] * w[0]
    return tuple(OC.to_fourier(st, H) for H in (H1, H2, H3))


def _rhs(nchi_k3_sign=1.0, nom_k1_sign=-1.0, swap=False):
    def rhs_terms(st, H1, H2, H3):
        K1, K3 = (st.K3, st.K1) if swap else (st.K1, st.K3)
        Nchi = -OC.apply_y(st.D1, 1j * st.K1 * H1 + nchi_k3_sign * 1j * st.K3 * H3) - st.K2 * H2
        Nom = 1j * K3 * H1 + nom_k1_sign * 1j * K1 * H3
        return Nchi * st.keep, Nom * st.keep
    return rhs_terms


def _vorticity_om1_flipped(st, S, u1, v, u3, du1, du3):
    om1 = du3 + 1j * st.K3 * v               # slip: sign of i k_3 v
    om3 = 1j * st.K1 * v - du1
    return om1, S["omega2"], om3


def _oblique_off(rate, rv, rw, prof):
    return (abs(rv - rate) > 2e-3 * abs(rate) or abs(rw - rate) > 2e-3 * abs(rate)
            or prof > 1e-3)


@pytest.mark.parametrize("name,attr,fn", [
    ("sign of u1 omega2 in H3", "nonlinear", _nonlinear_h3_flipped),
    ("sign of k3 H3 in N_chi", "rhs_terms", _rhs(nchi_k3_sign=-1.0)),
    ("sign of k1 H3 in N_omega2", "rhs_terms", _rhs(nom_k1_sign=1.0)),
    ("k1 and k3 swapped in N_omega2", "rhs_terms", _rhs(swap=True)),
])
def test_oblique_mode_pin_catches(monkeypatch, name, attr, fn):
    assert not _oblique_off(*pins.oblique_mode_rates())
    monkeypatch.setattr(OC, attr, fn)
    assert _oblique_off(*pins.oblique_mode_rates()), name


@pytest.fixture(scope="module")
def c1_state():
    st = OC.Setup(180, math.pi, math.pi / 2, 32, 49, 32, 1e-3)
    ic = SY.perturbed_poiseuille(st.y, 180, st.Lx, st.Lz, 32, 32, seed=7, amp=0.1)
    return st, OC.run(st, OC.initial_state(st, ic["v"], ic["omega2"], ic["U1"], ic["U3"]), 2)


def test_energy_pin_catches_a_quadratic_only_slip(monkeypatch, c1_state):
    """u_3 omega_2 in H_1 is a product of two perturbations: invisible to the linear
    pins, caught by the energy identity."""
    st, S = c1_state
    assert pins.energy_residual(st, S) < 1e-14
    monkeypatch.setattr(OC, "nonlinear", _nonlinear_h1_flipped)
    assert pins.energy_residual(st, S) > 1e-3


def test_vorticity_pin_catches_a_sign_slip(monkeypatch, c1_state):
    """omega_1 enters H only through perturbation products; its sign is caught by div omega = 0."""
    st, S = c1_state
    assert pins.vorticity_divergence(st, S) < 1e-13
    monkeypatch.setattr(OC, "vorticity", _vorticity_om1_flipped)
    assert pins.vorticity_divergence(st, S) > 1e-3
