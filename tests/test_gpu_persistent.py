"""Persistent work-list launches of a batch (CHAN_BATCH_PERSISTENT): one launch advances
each run by its own number of substeps, the launch's CTAs taking the blocks of any run whose
previous stage is done.  Each run's result must be bitwise the one of its own single-run
steps, for runs of different sizes at different RK3 phases, any counts (including none and
more than one launch holds); a launch whose polls run out (a stage made to need one
completion more than it can get) must come back as CHAN_ETIMEOUT with the context usable,
and the batch must step correctly again."""
import math

import numpy as np
import pytest

import synthetic as SY

pytestmark = pytest.mark.gpu

SHAPES = [(32, 49, 32, 180.0), (64, 97, 32, 395.0), (48, 49, 64, 550.0), (128, 33, 96, 395.0)]


def _make(chan, nx, ny, nz, re, prec):
    ch = chan.Channel(re, math.pi, math.pi / 2, nx, ny, nz, 5e-4, precision=prec)
    s0 = SY.perturbed_poiseuille(ch.grid(), re, math.pi, math.pi / 2, nx, nz, seed=nx + ny + nz, amp=0.1)
    ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    return ch


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_persistent_batch_is_bitwise_equal_to_per_run_steps(prec):
    import paper_1808_06461_b300 as chan
    lead = [0, 1, 2, 0]   # each run starts at its own RK3 phase
    alone = [_make(chan, *sh, prec) for sh in SHAPES]
    for ch, l in zip(alone, lead):
        if l:
            ch.step(l)
        ch.step(7)
        ch.step(5)
    runs = [_make(chan, *sh, prec) for sh in SHAPES]
    for ch, l in zip(runs, lead):
        if l:
            ch.step(l)
    b = chan.ChannelBatch(runs, persistent=True)
    assert b.persistent_grid() >= 148
    b.step(7)        # one launch of seven substeps of every run
    b.step(5)
    b.status()
    b.close()
    for a, p in zip(alone, runs):
        ga, gp = a.get_state(), p.get_state()
        for k in ("v", "omega2", "U1", "U3"):
            assert np.array_equal(ga[k], gp[k]), (prec, k)
        assert a.substeps() == p.substeps() and a.time() == p.time()


def test_a_wait_that_runs_out_is_reported_and_the_batch_recovers():
    import paper_1808_06461_b300 as chan
    runs = [_make(chan, *sh, 0) for sh in SHAPES[:3]]
    b = chan.ChannelBatch(runs, persistent=True)
    # run 1's z-inverse stage of the first substep needs one completion more than it has
    # items: the x-pass items of run 1 wait on it until 20000 polls (a few ms) run out
    b.set_wait(20000, hold_run=1, hold_stage=1)
    b.step(3)
    with pytest.raises(chan.ChanError) as e:
        b.status()
    assert e.value.code == chan.CHAN_ETIMEOUT
    b.status()       # the flag is cleared by the read
    # the context is usable: restore the default limit, fresh states, compare with per-run steps
    b.set_wait(1 << 23)
    fresh = [_make(chan, *sh, 0) for sh in SHAPES[:3]]
    for ch, f in zip(runs, fresh):
        g = f.get_state()
        ch.set_state(g["v"], g["omega2"], g["U1"], g["U3"])
        f.step(6)
    b.step(6)
    b.status()
    b.close()
    for a, p in zip(fresh, runs):
        ga, gp = a.get_state(), p.get_state()
        for k in ("v", "omega2", "U1", "U3"):
            assert np.array_equal(ga[k], gp[k]), k


def test_persistent_serving_alone_and_in_the_mix_are_identical():
    from paper_1808_06461_b300.serve import Request, Server, channel_factory, serving_dt

    def ic(r, y):
        return SY.perturbed_poiseuille(y, r.re_tau, r.Lx, r.Lz, r.Nx, r.Nz, seed=r.seed, amp=0.1)

    shapes = [(32, 49, 32, 180.0), (64, 49, 32, 395.0), (32, 97, 64, 550.0), (64, 49, 64, 180.0)]
    reqs = [Request(i, 0.0, re, math.pi, math.pi / 2, nx, ny, nz, serving_dt(re, math.pi, math.pi / 2, nx, nz),
                    31 + 4 * i, 300 + i, 3) for i, (nx, ny, nz, re) in enumerate(shapes)]
    alone, _ = Server(64 << 30, max_slots=1, factory=channel_factory(ic)).run(reqs)
    served, m = Server(64 << 30, max_slots=4, factory=channel_factory(ic), packed="persistent").run(reqs)
    assert m["packed"] == "persistent" and m["max_concurrency"] == 4
    for r in reqs:
        for k in ("v", "omega2", "U1", "U3"):
            assert np.array_equal(alone[r.rid][k], served[r.rid][k]), (r.rid, k)


@pytest.mark.parametrize("prec", [0, 3])
def test_runs_of_one_launch_advance_by_their_own_counts(prec):
    import paper_1808_06461_b300 as chan
    counts = [(7, 5), (12, 0), (0, 9), (50, 1)]   # 50 > 48: two launches for that run
    alone = [_make(chan, *sh, prec) for sh in SHAPES]
    for ch, ks in zip(alone, counts):
        for k in ks:
            if k:
                ch.step(k)
    runs = [_make(chan, *sh, prec) for sh in SHAPES]
    b = chan.ChannelBatch(runs, persistent=True)
    for q in range(2):
        b.step_each([ks[q] for ks in counts])
    b.status()
    b.close()
    for a, p, ks in zip(alone, runs, counts):
        ga, gp = a.get_state(), p.get_state()
        for k in ("v", "omega2", "U1", "U3"):
            assert np.array_equal(ga[k], gp[k]), (prec, ks, k)
        assert p.substeps() == sum(ks) and a.time() == p.time()


def test_persistent_batches_refuse_what_they_cannot_hold():
    import ctypes
    import paper_1808_06461_b300 as chan
    lib = chan.library()
    runs = [_make(chan, 32, 17, 32, 180.0, 0) for _ in range(17)]
    arr = (ctypes.c_void_p * 17)(*[c.h.value for c in runs])
    b = ctypes.c_void_p()
    # more than 16 runs in one persistent launch
    assert lib.chan_batch_create_ex(ctypes.byref(b), arr, 17, None, chan.CHAN_BATCH_PERSISTENT) == chan.CHAN_EINVAL
    assert not b.value
    # an unknown flag
    assert lib.chan_batch_create_ex(ctypes.byref(b), arr, 2, None, 2) == chan.CHAN_EINVAL
    # per-run counts and wait limits are checked
    pb = chan.ChannelBatch(runs[:2], persistent=True)
    with pytest.raises(chan.ChanError):
        pb.step_each([3, -1])
    with pytest.raises(chan.ChanError):
        pb.set_wait(0)
    pb.close()
    # the per-kernel batch has no persistent controls
    kb = chan.ChannelBatch(runs[:2])
    with pytest.raises(chan.ChanError):
        kb.step_each([3, 3])
    with pytest.raises(chan.ChanError):
        kb.set_wait(100)
    kb.status()
    kb.close()
    for c in runs:
        c.close()
