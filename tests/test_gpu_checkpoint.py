"""Checkpoint and restart: a run restarted from a checkpoint continues bitwise as the
original (mid RK3 step, with the kept implicit right-hand sides), in every precision;
a checkpoint of another box is refused."""
import math

import numpy as np
import pytest

import synthetic as SY

pytestmark = pytest.mark.gpu

CFG = (250.0, 2.0, 1.3, 24, 33, 36, 1e-3)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_restart_is_bitwise(prec):
    import paper_1808_06461_b300 as chan
    re, Lx, Lz, Nx, Ny, Nz, dt = CFG
    a = chan.Channel(*CFG, precision=prec)
    s0 = SY.perturbed_poiseuille(a.grid(), re, Lx, Lz, Nx, Nz, seed=8, amp=0.1)
    a.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    a.step(4)                       # mid RK3 step
    ck = a.checkpoint()
    t4 = a.time()
    a.step(7)
    ga = a.get_state()
    b = chan.Channel(*CFG, precision=prec)
    b.restore(ck)
    assert b.substeps() == 4 and b.time() == t4
    b.step(7)
    gb = b.get_state()
    for k in ("v", "omega2", "U1", "U3"):
        assert np.array_equal(ga[k], gb[k]), (prec, k)
    assert a.time() == b.time() and a.substeps() == b.substeps() == 11
    a.close()
    b.close()


def test_checkpoint_of_another_box_is_refused():
    import paper_1808_06461_b300 as chan
    re, Lx, Lz, Nx, Ny, Nz, dt = CFG
    a = chan.Channel(*CFG)
    s0 = SY.perturbed_poiseuille(a.grid(), re, Lx, Lz, Nx, Nz, seed=8, amp=0.1)
    a.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    ck = a.checkpoint()
    b = chan.Channel(re, Lx, Lz, Nx, Ny, Nz, 2 * dt)
    with pytest.raises(chan.ChanError) as e:
        b.restore(ck)
    assert e.value.code == chan.CHAN_EINVAL
    with pytest.raises(chan.ChanError):
        b.restore(np.zeros_like(ck))
    a.close()
    b.close()
