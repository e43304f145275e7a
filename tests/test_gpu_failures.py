"""Failure handling on the GPU, with faults injected on the host only (no device
trap, no bad address): non-finite input state, an allocation the device cannot
hold, calls out of order."""
import ctypes
import math

import numpy as np
import pytest

import synthetic as SY

pytestmark = pytest.mark.gpu


def _channel(chan):
    ch = chan.Channel(180.0, math.pi, math.pi / 2, 32, 49, 32, 1e-3)
    s0 = SY.perturbed_poiseuille(ch.grid(), 180.0, math.pi, math.pi / 2, 32, 32, seed=2, amp=0.1)
    return ch, s0


def test_nan_in_the_state_is_reported():
    import paper_1808_06461_b300 as chan
    ch, s0 = _channel(chan)
    U1 = s0["U1"].copy()
    U1[10] = np.nan                      # planted in a host-side copy of the mean profile
    ch.set_state(s0["v"], s0["omega2"], U1, s0["U3"])
    ch.step(3)
    with pytest.raises(chan.ChanError) as e:
        ch.stats()
    assert e.value.code == chan.CHAN_ENAN
    with pytest.raises(chan.ChanError) as e:
        ch.get_state()
    assert e.value.code == chan.CHAN_ENAN
    # the handle stays usable: a clean state steps and reads back
    ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    ch.step(3)
    assert np.isfinite(ch.get_state()["U1"]).all()


def test_allocation_beyond_the_device_is_an_error_not_a_fault():
    import paper_1808_06461_b300 as chan
    lib = chan.library()
    need = chan.footprint_bytes(768, 4097, 768, chan.CHAN_PREC_FP64)
    assert need > 300e9                  # more than the 288 GB (275,040 MiB) of HBM
    h = ctypes.c_void_p()
    rc = lib.chan_init(ctypes.byref(h), 180.0, math.pi, math.pi / 2, 768, 4097, 768, 1e-3)
    assert rc == chan.CHAN_ENOMEM and not h.value
    assert "cudaMalloc" in lib.chan_last_error(None).decode()
    ch, s0 = _channel(chan)              # the device is fine afterwards
    ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    ch.step(3)
    assert np.isfinite(ch.get_state()["v"]).all()


def test_calls_out_of_order():
    import paper_1808_06461_b300 as chan
    ch, _ = _channel(chan)
    for call in (lambda: ch.step(1), lambda: ch.stats(), lambda: ch.filter_stresses(0, 120, 60),
                 lambda: ch.get_state(), lambda: ch.autotune()):
        with pytest.raises(chan.ChanError) as e:
            call()
        assert e.value.code == chan.CHAN_ESTATE
