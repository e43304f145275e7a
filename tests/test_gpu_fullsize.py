"""Parity at the full Re_tau = 550, 384 x 257 x 384 workload, in the launch
configuration bench.py times (FP64, the library's kernels on a torch stream).

The oracle computes sampled outputs one by one: the dealiased H on sampled
x-z planes (the transforms are plane-local), and the whole substep for
sampled Fourier modes (the implicit solves are mode-local once the
non-linear terms of every plane are known; those are computed plane-chunk
by plane-chunk).  Properties that hold at any size (continuity, wall
conditions, flux, Hermitian symmetry) are checked over every mode.
"""
import copy
import math

import numpy as np
import pytest

import oracle as O
import synthetic as SY

pytestmark = pytest.mark.gpu

CFG = (550.0, 2 * math.pi, math.pi, 384, 257, 384, 2e-4)
TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def big():
    import torch
    import paper_1808_06461_b300 as chan
    st = O.Setup(*CFG)
    s0 = SY.turbulent_like(st.y, CFG[0], CFG[1], CFG[2], CFG[3], CFG[5], seed=1)
    ch = chan.Channel(*CFG, stream=torch.cuda.current_stream().cuda_stream)
    ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    S = O.initial_state(st, s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    return st, s0, S, ch


def _nonlinear_planes(st, S, vel, planes):
    u1, v, u3, du1, dv, du3 = vel
    om1 = du3[planes] - 1j * st.K3 * v[planes]
    om3 = 1j * st.K1 * v[planes] - du1[planes]
    p = [O.to_physical(st, F) for F in (u1[planes], v[planes], u3[planes], om1, S["omega2"][planes], om3)]
    H1 = p[1] * p[5] - p[2] * p[4]
    H2 = p[2] * p[3] - p[0] * p[5]
    H3 = p[0] * p[4] - p[1] * p[3]
    return [O.to_fourier(st, H) for H in (H1, H2, H3)]


def test_fullsize_nonlinear_sampled_planes(big):
    st, s0, S, ch = big
    H = ch.nonlinear()
    vel = O.velocities(st, S)
    planes = np.array([0, 1, 3, 64, 128, 200, 255, 256])
    ref = _nonlinear_planes(st, S, vel, planes)
    for f in range(3):
        assert rel(H[f][planes], ref[f]) < 1e-12, (f, rel(H[f][planes], ref[f]))


@pytest.fixture(scope="module")
def one_substep_ref(big):
    """The oracle's first substep on sampled modes (H of every plane, chunk by chunk)."""
    st, s0, S, ch = big
    vel = O.velocities(st, S)
    H = [np.zeros_like(S["v"]) for _ in range(3)]
    for c0 in range(0, st.Ny, 32):
        pl = np.arange(c0, min(st.Ny, c0 + 32))
        Hc = _nonlinear_planes(st, S, vel, pl)
        for k in range(3):
            H[k][pl] = Hc[k]
    Nchi, Nom = O.rhs_terms(st, *H)
    M = st.Nz * st.nxh
    rng = np.random.default_rng(0)
    sel = np.unique(np.concatenate([[1, 2, st.nxh, st.nxh + 1, M - 1], rng.integers(0, M, 250)]))
    sts = copy.copy(st)
    for k in ("K1", "K3", "K2", "keep"):
        setattr(sts, k, getattr(st, k).reshape(1, -1)[:, sel])
    sub = lambda F: F.reshape(st.Ny, 1, M)[:, :, sel]
    Ss = dict(S, v=sub(S["v"]), omega2=sub(S["omega2"]), chi=sub(S["chi"]),
              Nchi_prev=sub(S["Nchi_prev"]), Nom_prev=sub(S["Nom_prev"]))
    om, chi, v = O.channel.implicit_step(sts, Ss, sub(Nchi), sub(Nom), 0)
    U1, U3, f = O.channel.mean_flow_step(st, S, H[0][:, 0, 0].real, H[2][:, 0, 0].real, 0)
    return sub, dict(v=v, omega2=om, U1=U1, U3=U3)


@pytest.mark.parametrize("prec,tol", [(0, TOL), (2, TOL), (1, 1e-5)])
def test_fullsize_one_substep_sampled_modes(big, one_substep_ref, prec, tol):
    """One substep at full size against the oracle on sampled modes: FP64 and double-float
    at the 1e-10 bar, mixed (FP32 transforms) at 1e-5."""
    import torch
    import paper_1808_06461_b300 as chan
    st, s0, S, ch = big
    sub, ref = one_substep_ref
    if prec != 0:
        ch = chan.Channel(*CFG, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    ch.step(1)
    g = ch.get_state()
    if prec != 0:
        ch.close()
    assert rel(sub(g["v"]), ref["v"]) < tol
    assert rel(sub(g["omega2"]), ref["omega2"]) < tol
    assert rel(g["U1"], ref["U1"]) < tol
    assert np.abs(g["U3"] - ref["U3"]).max() < tol * np.abs(ref["U1"]).max()


def test_fullsize_invariants_after_substeps(big):
    st, s0, S, ch = big
    ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    ch.step(6)
    g = ch.get_state()
    Sg = dict(v=g["v"], omega2=g["omega2"], U1=g["U1"], U3=g["U3"])
    u1, v, u3, _, dv, _ = O.velocities(st, Sg)
    scale = np.abs(u1[:, :, 1:]).max()
    assert np.isfinite(g["v"]).all() and np.isfinite(g["omega2"]).all()
    assert O.divergence(st, Sg) < 1e-11 * scale
    assert np.abs(g["v"][[0, -1]]).max() < 1e-14 * scale
    assert np.abs(dv[[0, -1]]).max() < 1e-10 * scale
    assert abs(st.flux(g["U1"]) - st.flux(s0["U1"])) < 1e-13 * st.flux(s0["U1"])
    F = g["omega2"]
    for jz in (1, 2, 50, st.Nz // 2 - 1):
        assert np.abs(F[:, jz, 0] - np.conj(F[:, st.Nz - jz, 0])).max() < 1e-12 * np.abs(F).max()
    assert np.abs(F[:, st.Nz // 2, :]).max() == 0


@pytest.mark.parametrize("kind,p", [(0, (120.0, 60.0)), (1, (50.0, 50.0))])
def test_fullsize_filter_sampled_planes(big, kind, p):
    """ubar_i and tau_ij (Sec. 3.1) of the full workload on sampled planes.  The filter pass
    runs in slabs of 242 planes here (six products and nine outputs within 4 GiB): planes 241
    and 242 lie on either side of the slab boundary.  The filter is plane-local, so the oracle
    computes tau on those planes alone, from the full fields' products."""
    st, s0, S, ch = big
    g = ch.get_state()
    Sg = O.initial_state(st, g["v"], g["omega2"], g["U1"], g["U3"])
    ub, tau = ch.filter_stresses(kind, *p)
    planes = np.array([0, 1, 120, 241, 242, 243, 256])
    G = O.filter_transfer(st, kind, *p)
    u1, v, u3, _, _, _ = O.velocities(st, Sg)
    u = [u1[planes], v[planes], u3[planes]]
    ubr = [G * f for f in u]
    pu = [O.to_physical(st, f) for f in u]
    pb = [O.to_physical(st, f) for f in ubr]
    for f in range(3):
        assert rel(ub[f][planes], ubr[f]) < TOL, (f, rel(ub[f][planes], ubr[f]))
    for q, (i, j) in enumerate(O.PAIRS):
        ref = G * O.to_fourier(st, pu[i] * pu[j]) - O.to_fourier(st, pb[i] * pb[j])
        assert rel(tau[q][planes], ref) < TOL, (q, rel(tau[q][planes], ref))
