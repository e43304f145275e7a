"""A handle may keep no Helmholtz right-hand sides (chan_opts.keep_rhs = -1, two Fourier
fields less; the default for boxes past 150 GB): every substep then forms the
right-hand side of the implicit step with the B product (Appendix A, Eqs. (psi) and
(chi1)) instead of recovering B X from the previous solve's kept right-hand side.
Both forms are the same discrete operator, so the FP64 path still matches the oracle
at 1e-10 after 10 substeps, every mode agrees with the kept form to its own rounding,
and a restart without kept right-hand sides is bitwise."""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as SY

pytestmark = pytest.mark.gpu

CFG = (250.0, 2.0, 1.3, 24, 33, 36, 1e-3)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _ic(ch):
    re, Lx, Lz, Nx, Ny, Nz, dt = CFG
    return SY.perturbed_poiseuille(ch.grid(), re, Lx, Lz, Nx, Nz, seed=6, amp=0.1)


def test_fp64_without_kept_rhs_matches_the_oracle():
    import paper_1808_06461_b300 as chan
    ch = chan.Channel(*CFG, keep_rhs=-1)
    s0 = _ic(ch)
    ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    ch.step(10)
    g = ch.get_state()
    ch.close()
    st = O.Setup(*CFG)
    ref = O.run(st, O.initial_state(st, s0["v"], s0["omega2"], s0["U1"], s0["U3"]), 10)
    for k in ("v", "omega2", "U1", "U3"):
        assert rel(g[k], ref[k]) < 1e-10, (k, rel(g[k], ref[k]))


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 1e-6), (2, 1e-12), (3, 1e-6)])
def test_without_kept_rhs_agrees_with_the_kept_form(prec, tol):
    import paper_1808_06461_b300 as chan
    out = []
    for keep in (1, -1):
        ch = chan.Channel(*CFG, precision=prec, keep_rhs=keep)
        s0 = _ic(ch)
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        ch.step(7)
        out.append(ch.get_state())
        ch.close()
    for k in ("v", "omega2", "U1"):
        assert rel(out[1][k], out[0][k]) < tol, (prec, k, rel(out[1][k], out[0][k]))


@pytest.mark.parametrize("prec", [0, 3])
def test_restart_without_kept_rhs_is_bitwise(prec):
    import paper_1808_06461_b300 as chan
    a = chan.Channel(*CFG, precision=prec, keep_rhs=-1)
    s0 = _ic(a)
    a.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    a.step(4)
    ck = a.checkpoint()
    a.step(5)
    ga = a.get_state()
    b = chan.Channel(*CFG, precision=prec, keep_rhs=-1)
    b.restore(ck)
    b.step(5)
    gb = b.get_state()
    for k in ("v", "omega2", "U1", "U3"):
        assert np.array_equal(ga[k], gb[k]), (prec, k)
    c = chan.Channel(*CFG, precision=prec)   # keeps them: a checkpoint without them is refused
    with pytest.raises(chan.ChanError):
        c.restore(ck)
    for h in (a, b, c):
        h.close()
