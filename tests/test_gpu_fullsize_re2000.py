"""The Re_tau = 2000 relaxed-resolution workload (Lx = 2 pi, Lz = pi, 1536 x 633 x
1152, dt = 5e-5) in mixed precision, the mode it is run in: about 147 GB on the
device, with the transforms in slabs, no kept Helmholtz right-hand sides, and the
implicit-step tables and Poisson factors recomputed each substep into work fields
that are dead from the non-linear terms to the Poisson step (all chosen
automatically for a box of this size).

The oracle computes the dealiased non-linear term on sampled x-z planes
(padded 2304 x 1728 transforms); the velocities it needs come from the
wall-normal operators applied mode chunk by mode chunk, so the host never holds
more than a few full fields.  After three substeps: continuity on sampled
modes, wall conditions, the mass flux and the Hermitian symmetry of the kx = 0
plane over every mode.
"""
import copy
import math

import numpy as np
import pytest

import oracle as O
import synthetic as SY

pytestmark = pytest.mark.gpu

CFG = (2000.0, 2 * math.pi, math.pi, 1536, 633, 1152, 5e-5)
PLANES = np.array([0, 1, 3, 150, 316, 500, 631, 632])


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _sub_setup(st, sel):
    """The oracle's set-up restricted to the stored modes sel (flattened kz, kx indices)."""
    sts = copy.copy(st)
    for k in ("K1", "K3", "K2", "keep"):
        setattr(sts, k, getattr(st, k).reshape(1, -1)[:, sel])
    return sts


def _velocities_on(st, v, om, U1, U3, sel):
    """The oracle's velocities on the modes sel.  Its (0, 0) slot carries the mean profiles,
    so mode 0 leads the subset (and is dropped again when sel does not hold it)."""
    M = st.Nz * st.nxh
    lead = sel[0] != 0
    full = np.concatenate([[0], sel]) if lead else sel
    sub = lambda F: F.reshape(st.Ny, 1, M)[:, :, full]
    out = O.velocities(_sub_setup(st, full), dict(v=sub(v), omega2=sub(om), U1=U1, U3=U3))
    return tuple(f[:, :, 1:] if lead else f for f in out)


def oracle_planes(cfg, planes, seed):
    """(set-up, initial field, the oracle's H on the given planes), velocities chunk by chunk."""
    st = O.Setup(*cfg)
    s0 = SY.turbulent_like(st.y, cfg[0], cfg[1], cfg[2], cfg[3], cfg[5], seed=seed)
    PLANES = planes
    M = st.Nz * st.nxh
    fields = [np.empty((len(PLANES), M), dtype=np.complex128) for _ in range(6)]
    for c0 in range(0, M, 32768):
        sel = np.arange(c0, min(M, c0 + 32768))
        u1, v, u3, du1, dv, du3 = _velocities_on(st, s0["v"], s0["omega2"], s0["U1"], s0["U3"], sel)
        K1 = st.K1.reshape(-1)[sel]
        K3 = st.K3.reshape(-1)[sel]
        om2 = s0["omega2"].reshape(st.Ny, M)[:, sel]
        vals = (u1[PLANES, 0], v[PLANES, 0], u3[PLANES, 0], du3[PLANES, 0] - 1j * K3 * v[PLANES, 0],
                om2[PLANES], 1j * K1 * v[PLANES, 0] - du1[PLANES, 0])
        for f in range(6):
            fields[f][:, sel] = vals[f]
    shp = (len(PLANES), st.Nz, st.nxh)
    p = [O.to_physical(st, F.reshape(shp)) for F in fields]
    H = [O.to_fourier(st, h) for h in (p[1] * p[5] - p[2] * p[4], p[2] * p[3] - p[0] * p[5],
                                      p[0] * p[4] - p[1] * p[3])]
    return st, s0, H


@pytest.fixture(scope="module")
def ref():
    return oracle_planes(CFG, PLANES, seed=4)


def test_re2000_mixed_nonlinear_sampled_planes_and_invariants(ref):
    import torch
    import paper_1808_06461_b300 as chan
    st, s0, Href = ref
    ch = chan.Channel(*CFG, precision=chan.CHAN_PREC_MIXED, stream=torch.cuda.current_stream().cuda_stream)
    try:
        assert ch.device_bytes() < 150e9
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        H = ch.nonlinear()
        for f in range(3):
            assert rel(H[f][PLANES], Href[f]) < 2e-5, (f, rel(H[f][PLANES], Href[f]))
        del H
        ch.step(3)
        g = ch.get_state()
        # the box filter of width 100 wall units through the filter pass's own slabs (20 planes
        # of 633, the last one ragged): the second-order identity <u_i u_j> = <ubar_i ubar_j> +
        # <tau_ij> on every plane (the filtered rows come from the products of the fluctuations)
        ch.filter_stresses(1, 100.0, 100.0, want=False)
        out = ch.stats()[0]
    finally:
        ch.close()
    scale = np.abs(out[2:8]).max()
    assert np.abs(out[2:8] - out[8:14] - out[14:20]).max() < 1e-6 * scale
    assert (out[14:17] > -1e-6 * scale).all()
    assert np.isfinite(g["U1"]).all()
    M = st.Nz * st.nxh
    rng = np.random.default_rng(1)
    sel = np.unique(np.concatenate([[1, 2, st.nxh, st.nxh + 1, M - 1], rng.integers(0, M, 400)]))
    u1, v, u3, _, dv, _ = _velocities_on(st, g["v"], g["omega2"], g["U1"], g["U3"], sel)
    sts = _sub_setup(st, sel)
    div = 1j * sts.K1 * u1 + dv + 1j * sts.K3 * u3
    scale = np.abs(u1).max()
    assert np.abs(div).max() < 1e-11 * scale
    assert np.abs(dv[[0, -1]]).max() < 1e-10 * scale
    assert np.abs(g["v"][[0, -1]]).max() < 1e-14 * np.abs(g["v"]).max() * 1e3
    assert abs(st.flux(g["U1"]) - st.flux(s0["U1"])) < 1e-13 * st.flux(s0["U1"])
    F = g["omega2"]
    fmax = np.abs(F).max()
    for jz in (1, 2, 200, st.Nz // 2 - 1):
        assert np.abs(F[:, jz, 0] - np.conj(F[:, st.Nz - jz, 0])).max() < 1e-7 * fmax
    assert np.abs(F[:, st.Nz // 2, :]).max() == 0
