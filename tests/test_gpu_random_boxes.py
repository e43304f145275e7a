"""Parity with the oracle on seeded random boxes: sizes from the whole admissible set
(Nx even and 2^a 3^b, Nz a multiple of 4 and 2^a 3^b, Ny odd), random Reynolds numbers
and periods, the serving time step.  FP64 and double-float at the 1e-10 bar after 10
substeps, mixed at the FP32 level."""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as SY

pytestmark = pytest.mark.gpu


def _boxes(n, seed):
    from paper_1808_06461_b300.serve import serving_dt
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.choice([2, 4, 6, 8, 12, 16, 18, 24, 32, 36]))
        nz = int(rng.choice([4, 8, 12, 16, 24, 32, 36, 48]))
        ny = int(rng.choice(np.arange(9, 66, 2)))
        re = float(rng.uniform(100.0, 600.0))
        lx, lz = float(rng.uniform(1.0, 7.0)), float(rng.uniform(0.5, 3.5))
        out.append((re, lx, lz, nx, ny, nz, serving_dt(re, lx, lz, nx, nz)))
    return out


BOXES = _boxes(6, 2026)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.fixture(scope="module")
def refs():
    out = []
    for cfg in BOXES:
        st = O.Setup(*cfg)
        s0 = SY.perturbed_poiseuille(st.y, cfg[0], cfg[1], cfg[2], cfg[3], cfg[5], seed=3, amp=0.1)
        S = O.initial_state(st, s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        out.append((s0, O.run(st, S, 10)))
    return out


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-10), (1, 1e-5), (3, 1e-5)])
@pytest.mark.parametrize("k", range(len(BOXES)))
def test_random_box_ten_substeps(refs, k, prec, tol):
    import paper_1808_06461_b300 as chan
    cfg = BOXES[k]
    s0, ref = refs[k]
    ch = chan.Channel(*cfg, precision=prec)
    ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    ch.step(10)
    g = ch.get_state()
    ch.close()
    for f in ("v", "omega2", "U1"):
        assert rel(g[f], ref[f]) < tol, (cfg, prec, f, rel(g[f], ref[f]))
