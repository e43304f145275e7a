"""Parity at the Re_tau = 1000, 768 x 385 x 768 workload (Lx = 2 pi, Lz = pi,
dt = 1e-4), in FP64, double-float and the two mixed modes the workload is run in.

The dealiased non-linear term is plane-local, so the oracle computes it on
sampled x-z planes (padded 1152 x 1152 transforms) from the same state.
Properties that hold at any size (continuity, wall conditions, the mass
flux, Hermitian symmetry of the kx = 0 plane) are checked over every mode
after three substeps.
"""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as SY

pytestmark = pytest.mark.gpu

CFG = (1000.0, 2 * math.pi, math.pi, 768, 385, 768, 1e-4)
PLANES = np.array([0, 1, 2, 96, 192, 300, 383, 384])


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def ref():
    st = O.Setup(*CFG)
    s0 = SY.turbulent_like(st.y, CFG[0], CFG[1], CFG[2], CFG[3], CFG[5], seed=3)
    S = O.initial_state(st, s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    u1, v, u3, du1, dv, du3 = O.velocities(st, S)
    om1 = du3[PLANES] - 1j * st.K3 * v[PLANES]
    om3 = 1j * st.K1 * v[PLANES] - du1[PLANES]
    p = [O.to_physical(st, F) for F in (u1[PLANES], v[PLANES], u3[PLANES], om1, S["omega2"][PLANES], om3)]
    H = [O.to_fourier(st, h) for h in (p[1] * p[5] - p[2] * p[4], p[2] * p[3] - p[0] * p[5],
                                      p[0] * p[4] - p[1] * p[3])]
    return st, s0, H


# FP64: both sides evaluate the same dealiased products in FP64 (rounding order only);
# double-float: pair transforms (~2^-47 per operation); mixed modes: FP32 transforms and
# products, the state and wall-normal operators in FP64 (mode 1) or pairs (mode 3).
# hsym: the kx = 0 plane is Hermitian in kz up to the rounding of the z transforms of
# real rows (unit roundoff 1.1e-16 in FP64, 6e-8 in FP32), entering through dt N (|N| up
# to 1e3 at the high wavenumbers) over three substeps; the x-pass drops the imaginary part
# of the kx = 0 column each substep, so the departure does not accumulate.
@pytest.mark.parametrize("prec,tol,hsym", [(0, 1e-12, 1e-12), (2, 1e-11, 1e-11), (1, 2e-5, 1e-7), (3, 2e-5, 1e-7)])
def test_re1000_nonlinear_sampled_planes_and_invariants(ref, prec, tol, hsym):
    import torch
    import paper_1808_06461_b300 as chan
    st, s0, Href = ref
    ch = chan.Channel(*CFG, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    try:
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        H = ch.nonlinear()
        for f in range(3):
            assert rel(H[f][PLANES], Href[f]) < tol, (prec, f, rel(H[f][PLANES], Href[f]))
        del H
        ch.step(3)
        g = ch.get_state()
    finally:
        ch.close()
    Sg = dict(v=g["v"], omega2=g["omega2"], U1=g["U1"], U3=g["U3"])
    u1, v, u3, _, dv, _ = O.velocities(st, Sg)
    scale = np.abs(u1[:, :, 1:]).max()
    assert np.isfinite(g["v"]).all() and np.isfinite(g["omega2"]).all()
    assert O.divergence(st, Sg) < 1e-11 * scale
    assert np.abs(g["v"][[0, -1]]).max() < 1e-14 * scale
    assert np.abs(dv[[0, -1]]).max() < 1e-10 * scale
    assert abs(st.flux(g["U1"]) - st.flux(s0["U1"])) < 1e-13 * st.flux(s0["U1"])
    F = g["omega2"]
    for jz in (1, 2, 100, st.Nz // 2 - 1):
        assert np.abs(F[:, jz, 0] - np.conj(F[:, st.Nz - jz, 0])).max() < hsym * np.abs(F).max()
    assert np.abs(F[:, st.Nz // 2, :]).max() == 0
