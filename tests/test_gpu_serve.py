"""Serving on the GPU: graph replay, footprint, and results alone vs in the mix."""
import math

import numpy as np
import pytest

import synthetic as SY

pytestmark = pytest.mark.gpu


def _ic(r, y):
    return SY.perturbed_poiseuille(y, r.re_tau, r.Lx, r.Lz, r.Nx, r.Nz, seed=r.seed, amp=0.1)


def test_graph_replay_is_bitwise_equal_to_single_launches():
    import paper_1808_06461_b300 as chan
    out = []
    for graph in (False, True):
        ch = chan.Channel(180.0, math.pi, math.pi / 2, 32, 49, 32, 1e-3)
        ch.set_graph(graph)
        s0 = SY.perturbed_poiseuille(ch.grid(), 180.0, math.pi, math.pi / 2, 32, 32, seed=9, amp=0.1)
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        ch.step(1)     # start off a step boundary: single launches, then graph steps, then a tail
        ch.step(13)
        out.append((ch.get_state(), ch.time(), ch.substeps()))
        ch.close()
    (a, ta, na), (b, tb, nb) = out
    for k in ("v", "omega2", "U1", "U3"):
        assert np.array_equal(a[k], b[k]), k
    assert ta == tb and na == nb == 14


def test_footprint_matches_allocation():
    import paper_1808_06461_b300 as chan
    for prec in (chan.CHAN_PREC_FP64, chan.CHAN_PREC_MIXED, chan.CHAN_PREC_F64X, chan.CHAN_PREC_MIXED_DF):
        ch = chan.Channel(395.0, math.pi, math.pi / 2, 64, 97, 32, 1e-3, precision=prec)
        s0 = SY.perturbed_poiseuille(ch.grid(), 395.0, math.pi, math.pi / 2, 64, 32, seed=1, amp=0.1)
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        ch.filter_stresses(0, 120.0, 60.0, want=False)
        assert ch.device_bytes() == chan.footprint_bytes(64, 97, 32, prec)
        ch.close()


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_results_alone_and_in_the_mix_are_identical(prec):
    """Each run's final state is bitwise the same served alone (one slot) or in a mix (four slots)."""
    from paper_1808_06461_b300.serve import Request, Server, channel_factory, serving_dt
    shapes = [(32, 49, 32, 180.0), (64, 49, 32, 395.0), (32, 97, 64, 550.0), (64, 49, 64, 180.0)]
    reqs = [Request(i, 0.0, re, math.pi, math.pi / 2, nx, ny, nz, serving_dt(re, math.pi, math.pi / 2, nx, nz),
                    30 + 3 * i, 100 + i, prec) for i, (nx, ny, nz, re) in enumerate(shapes)]
    alone, m1 = Server(64 << 30, max_slots=1, factory=channel_factory(_ic)).run(reqs)
    mixed, m2 = Server(64 << 30, max_slots=4, factory=channel_factory(_ic)).run(reqs)
    assert m1["max_concurrency"] == 1 and m2["max_concurrency"] == 4
    for r in reqs:
        for k in ("v", "omega2", "U1", "U3"):
            assert np.array_equal(alone[r.rid][k], mixed[r.rid][k]), (r.rid, k)
        assert np.isfinite(mixed[r.rid]["v"]).all()


def test_packed_batch_step_is_bitwise_equal_to_per_run_steps():
    import paper_1808_06461_b300 as chan
    shapes = [(32, 49, 32, 180.0), (64, 97, 32, 395.0), (48, 49, 64, 550.0)]

    def make(nx, ny, nz, re):
        ch = chan.Channel(re, math.pi, math.pi / 2, nx, ny, nz, 5e-4)
        s0 = SY.perturbed_poiseuille(ch.grid(), re, math.pi, math.pi / 2, nx, nz, seed=nx + ny, amp=0.1)
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        return ch

    alone = [make(*sh) for sh in shapes]
    for ch in alone:
        ch.step(7)
        ch.step(5)
    packed = [make(*sh) for sh in shapes]
    b = chan.ChannelBatch(packed)
    b.step(7)        # two graph-replayed RK3 steps and one single substep
    b.step(5)        # two substeps to the next step boundary, then one graph step
    b.close()
    for a, p in zip(alone, packed):
        ga, gp = a.get_state(), p.get_state()
        for k in ("v", "omega2", "U1", "U3"):
            assert np.array_equal(ga[k], gp[k]), k
        assert a.substeps() == p.substeps() == 12 and a.time() == p.time()


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_packed_serving_alone_and_in_the_mix_are_identical(prec):
    from paper_1808_06461_b300.serve import Request, Server, channel_factory, serving_dt
    shapes = [(32, 49, 32, 180.0), (64, 49, 32, 395.0), (32, 97, 64, 550.0), (64, 49, 64, 180.0)]
    reqs = [Request(i, 0.0, re, math.pi, math.pi / 2, nx, ny, nz, serving_dt(re, math.pi, math.pi / 2, nx, nz),
                    31 + 4 * i, 200 + i, prec) for i, (nx, ny, nz, re) in enumerate(shapes)]
    alone, _ = Server(64 << 30, max_slots=1, factory=channel_factory(_ic)).run(reqs)
    packed, m = Server(64 << 30, max_slots=4, factory=channel_factory(_ic), packed=True).run(reqs)
    assert m["packed"] and m["max_concurrency"] == 4
    for r in reqs:
        for k in ("v", "omega2", "U1", "U3"):
            assert np.array_equal(alone[r.rid][k], packed[r.rid][k]), (r.rid, k)


def test_autotuned_shapes_leave_results_unchanged():
    import paper_1808_06461_b300 as chan
    out = []
    for tune in (False, True):
        ch = chan.Channel(395.0, math.pi, math.pi / 2, 64, 49, 96, 1e-3)
        s0 = SY.perturbed_poiseuille(ch.grid(), 395.0, math.pi, math.pi / 2, 64, 96, seed=4, amp=0.1)
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        if tune:
            kb, nt, yt = ch.autotune()
            assert kb in (1, 2, 4, 8, 16) and nt in (96, 128, 144, 160, 192, 256, 288, 384, 512) and yt in (0, 1)
        ch.step(6)
        out.append(ch.get_state())
        ch.close()
    for k in ("v", "omega2", "U1", "U3"):
        assert np.array_equal(out[0][k], out[1][k]), k
